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
// The batched contraction is the split-TF32 kernel of gemm_tf32x3.cu driven by
// a device-side tile list: tiles of all transforms come from one dynamic queue,
// and the TMA producer chooses the factor source per tile.  A tile's B operand
// is up to eight 32-line segments, each from any (transform, l) group, so the
// narrow groups of one l (2(2l+1) lines each) from many transforms fill one
// 256-column MMA against one shared slab of T_l.  The batch owns its workspace
// and tensor maps, so a whole step can be captured into one CUDA graph
// (dsbt_batch_capture_kinetic).  An autotuner times the tile order
// (transform-major; l-major; l-major with row tiles interleaved across
// transforms; the same with segments of different transforms packed into one
// tile) and the column-tile width (128, 192, 256 lines) on the batch's own
// shapes at creation and keeps the fastest.
#include <math.h>

#include <string.h>

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
constexpr int SEG = 32;            // lines per B segment (one TMA box)
constexpr int SEG_MAX = BN_MAX / SEG;
constexpr int STAGES = 2;
constexpr int KC = 4;
constexpr int EPI_WARPS = 8;
constexpr int QS = 4;
constexpr int A_BYTES = BM * BK * 4;
constexpr int B_BYTES = BN_MAX * BK * 4;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int CROWS = 32;   // rows of the per-N tables (>= every completion-row count)
constexpr int kOrders = 4;  // tile orders offered to the autotuner

struct BGroup {
    int t, l, N, nl;   // transform, angular momentum, grid, real lines
    int bline0;        // first line of the group in the transform's planar buffers
    int cidx;          // distinct-N index of the per-N tables
    long long uoff;    // complex-element offset of the group's first channel (caller layout)
};

struct KR {
    int a0, a1, b0, b1, up;
    __device__ __forceinline__ int count() const { return (a1 - a0) + (b1 - b0); }
    __device__ __forceinline__ int at(int i) const {
        if (up) return (i < a1 - a0) ? (a0 + i) : (b0 + i - (a1 - a0));
        const int nb = b1 - b0;
        return (i < nb) ? (b1 - 1 - i) : (a1 - 1 - (i - nb));
    }
};

// K blocks of a tile: the forward T_l is dense in its completion rows (n < nx)
// and lower triangular below; T_l^T is dense in its first nx columns and upper
// triangular.
__device__ __forceinline__ KR kranges(int dir, int rt, int nx, int KB) {
    KR k;
    const int r0 = rt * BM;
    k.up = 1;
    k.a0 = 0;
    k.b0 = k.b1 = 0;
    if (r0 < nx) { k.a1 = KB; return k; }
    if (dir > 0) { k.a1 = min(KB, (r0 + BM) / BK); return k; }
    k.a1 = (nx + BK - 1) / BK;
    k.b0 = max(k.a1, r0 / BK);
    k.b1 = KB;
    return k;
}

// One output tile: rows [rt BM, rt BM + BM) of T_l (forward) or T_l^T
// (inverse) against up to SEG_MAX segments of SEG lines.  A segment is lines
// [c, c + SEG) of one (transform, l) group; lines past the group's end are
// computed and discarded.  Segments of one tile may come from different
// transforms.  The rows of the shared factors a forward tile with rt >= 1
// reads do not depend on N; a forward tile with rt = 0 reads per-N rows and
// holds one grid.  An inverse tile may hold several grids ("classes", N
// descending, contiguous): its K range ends at the largest N (the B operand of
// a smaller grid reads zeros past its own N through the tensor map bounds),
// and K block 0, which comes from each grid's own per-N table, runs as one
// sub-step per class on that class's columns.
struct __align__(16) PTile {
    int l, rt, N, cidx;   // N: grid of the K range, cidx: per-N tables of a one-grid tile
    int nseg, ncls, pad0, pad1;
    int g[SEG_MAX];       // group of each segment
    int c[SEG_MAX];       // first line of the segment in its group
    unsigned char cend[SEG_MAX];   // one past the last segment of each class
};

// Steps of one tile: K blocks ascending, with K block 0 (when in range) split
// into ns sub-steps, one per class of an inverse tile.  The main accumulator
// restarts at chunk boundaries: the first chunk holds the sub-steps and the
// next KC - 1 K blocks, later chunks KC K blocks, so no column accumulates
// more than KC K blocks in one chunk.
struct Steps {
    KR kr;
    int ns, nsteps, c0len;
    bool kb0;
    __device__ __forceinline__ int kb(int i) const {
        if (!kb0) return kr.at(i);
        return (i < ns) ? 0 : kr.at(i - ns + 1);
    }
    __device__ __forceinline__ int chunk_end(int start) const {
        return min(nsteps, start == 0 ? c0len : start + KC);
    }
};

__device__ __forceinline__ Steps make_steps(int dir, const PTile& tl) {
    Steps sp;
    sp.kr = kranges(dir, tl.rt, n_extra(tl.l), tl.N / BK);
    const int n = sp.kr.count();
    sp.kb0 = n > 0 && sp.kr.at(0) == 0;
    sp.ns = (sp.kb0 && dir < 0) ? tl.ncls : 1;
    sp.nsteps = sp.kb0 ? n - 1 + sp.ns : n;
    sp.c0len = sp.kb0 ? sp.ns + KC - 1 : KC;
    return sp;
}

// Segments [s0, s1) a step reads: one class in an inverse tile's K block 0
// sub-steps, else all.
__device__ __forceinline__ void step_segments(int dir, const PTile& tl, const Steps& sp, int i, int* s0, int* s1) {
    if (dir < 0 && sp.kb0 && i < sp.ns) {
        *s0 = i == 0 ? 0 : tl.cend[i - 1];
        *s1 = tl.cend[i];
    } else {
        *s0 = 0;
        *s1 = tl.nseg;
    }
}

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

// Per-transform B maps: a_hi, a_lo, b_hi, b_lo with boxes of 32, 64 and 128
// lines (index 4 * log2(lines / 32) + buffer), so runs of 2 or 4 contiguous
// segments of one group move with one TMA load per buffer.
struct __align__(64) TMaps {
    CUtensorMap m[12];
};

enum : int { kModeUserC64 = 0, kModeSplit = 1, kModePlanar = 2 };

__global__ void __launch_bounds__(NTHREADS, 1)
k_contract_batch(const __grid_constant__ CUtensorMap tF_hi, const __grid_constant__ CUtensorMap tF_lo,
                 const __grid_constant__ CUtensorMap tF96_hi, const __grid_constant__ CUtensorMap tF96_lo,
                 const __grid_constant__ CUtensorMap tI_hi, const __grid_constant__ CUtensorMap tI_lo,
                 const PTile* __restrict__ tiles, int total, const BGroup* __restrict__ groups,
                 const BTrans* __restrict__ trans, const TMaps* __restrict__ tmaps, const BMaps* __restrict__ cmaps,
                 int Nmax, int dir, int mode, float2* __restrict__ out_user, unsigned* status, uint32_t spin,
                 int* sched) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stage_base = smem;
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* main_full = empty + STAGES;
    uint64_t* main_empty = main_full + 1;
    uint64_t* tq_full = main_empty + 1;
    uint64_t* tq_empty = tq_full + QS;
    uint64_t* drain_bar = tq_empty + QS;    // the MMA issuer's exit drain
    int* tile_q = (int*)(drain_bar + 1);
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
        mbar_init(drain_bar, 1);
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
        __shared__ const CUtensorMap* mseg[SEG_MAX];   // per segment: 32-line B map, first line and
        __shared__ int yseg[SEG_MAX];                   // the contiguous run of segments it starts
        __shared__ int rseg[SEG_MAX];
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            StageLedger led;
            int qslot = 0;
            uint32_t qphase = 0;
            while (ok) {
                if (!mbar_wait(&tq_empty[qslot], qphase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                int t = atomicAdd(sched, 1);
                if (t >= total) t = -1;
                tile_q[qslot] = t;
                mbar_arrive(&tq_full[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (t < 0) break;
                const PTile& tl = tiles[t];
                const int l = tl.l, rt = tl.rt, nseg = tl.nseg;
                const Steps sp = make_steps(dir, tl);
                for (int s = 0; s < nseg; ++s) {
                    const BGroup& G = groups[tl.g[s]];
                    mseg[s] = &tmaps[G.t].m[dir > 0 ? 0 : 2];   // hi map; lo map follows it
                    yseg[s] = G.bline0 + tl.c[s];
                }
                for (int s = nseg - 1; s >= 0; --s)   // segments s, s+1, ... of one group, contiguous
                    rseg[s] = (s + 1 < nseg && tl.g[s + 1] == tl.g[s] && tl.c[s + 1] == tl.c[s] + SEG)
                                  ? rseg[s + 1] + 1 : 1;
                for (int i = 0; i < sp.nsteps; ++i) {
                    const int kb = sp.kb(i);
                    int s0, s1;
                    step_segments(dir, tl, sp, i, &s0, &s1);
                    if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                    unsigned char* sb = stage_base + stage * STAGE_BYTES;
                    mbar_expect_tx(&full[stage], 2 * A_BYTES + 2 * (s1 - s0) * SEG * BK * 4);
                    led.arm(stage, phase);
                    if (dir > 0) {
                        if (rt == 0) {   // rows 0..31 from the per-N table, 32..127 shared
                            const int cidx = tl.cidx;
                            tma_load_2d(sb, &cmaps[cidx].m[0], &full[stage], kb * BK, l * CROWS);
                            tma_load_2d(sb + A_BYTES, &cmaps[cidx].m[1], &full[stage], kb * BK, l * CROWS);
                            tma_load_2d(sb + CROWS * 128, &tF96_hi, &full[stage], kb * BK, l * Nmax + CROWS);
                            tma_load_2d(sb + A_BYTES + CROWS * 128, &tF96_lo, &full[stage], kb * BK,
                                        l * Nmax + CROWS);
                        } else {
                            tma_load_2d(sb, &tF_hi, &full[stage], kb * BK, l * Nmax + rt * BM);
                            tma_load_2d(sb + A_BYTES, &tF_lo, &full[stage], kb * BK, l * Nmax + rt * BM);
                        }
                    } else {
                        if (kb == 0) {      // K block 0 (rows n < 32 of T) from the class's per-N table
                            const BGroup& G = groups[tl.g[s0]];
                            tma_load_2d(sb, &cmaps[G.cidx].m[2], &full[stage], 0, l * G.N + rt * BM);
                            tma_load_2d(sb + A_BYTES, &cmaps[G.cidx].m[3], &full[stage], 0, l * G.N + rt * BM);
                        } else {
                            tma_load_2d(sb, &tI_hi, &full[stage], kb * BK, l * Nmax + rt * BM);
                            tma_load_2d(sb + A_BYTES, &tI_lo, &full[stage], kb * BK, l * Nmax + rt * BM);
                        }
                    }
                    for (int s = s0; s < s1;) {
                        const int run = min(rseg[s], s1 - s);
                        const int len = run >= 4 ? 4 : (run >= 2 ? 2 : 1);   // segments in this load
                        const CUtensorMap* m = mseg[s] + (len == 4 ? 8 : (len == 2 ? 4 : 0));
                        tma_load_2d(sb + 2 * A_BYTES + s * SEG * 128, m, &full[stage], kb * BK, yseg[s]);
                        tma_load_2d(sb + 2 * A_BYTES + B_BYTES + s * SEG * 128, m + 1, &full[stage], kb * BK,
                                    yseg[s]);
                        s += len;
                    }
                    if (++stage == STAGES) { stage = 0; phase ^= 1; }
                }
            }
            led.drain(full, STAGES, status);   // copies still in flight after an abort
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
                if (!mbar_wait(&tq_full[qslot], qphase, abort_flag, status, spin)) break;
                const int t = ((volatile int*)tile_q)[qslot];
                mbar_arrive(&tq_empty[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (t < 0) break;
                const PTile& tl = tiles[t];
                const Steps sp = make_steps(dir, tl);
                const uint32_t idesc_all = idesc_tf32(BM, tl.nseg * SEG);
                for (int c0 = 0; c0 < sp.nsteps && ok;) {
                    const int c1 = sp.chunk_end(c0);
                    // Inside a tile (c0 > 0: a full-width K block, never a sub-step), the
                    // first step's correction products go out before the wait for the
                    // epilogue to drain the main accumulator.
                    const bool pre = c0 > 0;
                    if (pre) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, status, spin)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(stage_base + stage * STAGE_BYTES);
                        const uint32_t sb_hi = sa + 2 * A_BYTES;
#pragma unroll
                        for (int ks = 0; ks < BK / 8; ++ks) {
                            const uint32_t off = ks * 32;
                            const uint64_t dah = sdesc_sw128(sa + off), dal = sdesc_sw128(sa + A_BYTES + off);
                            const uint64_t dbh = sdesc_sw128(sb_hi + off), dbl = sdesc_sw128(sb_hi + B_BYTES + off);
                            mma_tf32(d_corr, dah, dbl, idesc_all, 1);
                            mma_tf32(d_corr, dal, dbh, idesc_all, 1);
                        }
                    }
                    if (!mbar_wait(main_empty, mphase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                    mphase ^= 1;
                    tc_fence_after();
                    for (int i = c0; i < c1; ++i) {
                        const bool early = pre && i == c0;   // correction products already issued
                        int s0, s1;
                        step_segments(dir, tl, sp, i, &s0, &s1);
                        // first write of these columns in this chunk (main) / in this tile (correction)
                        const bool sub = s1 - s0 != tl.nseg;
                        const uint32_t fresh_main = (i == c0 || sub) ? 0u : 1u;
                        const uint32_t fresh_corr = (i == 0 || sub) ? 0u : 1u;
                        const uint32_t idesc = sub ? idesc_tf32(BM, (s1 - s0) * SEG) : idesc_all;
                        const uint32_t col0 = (uint32_t)(s0 * SEG);
                        if (!early) {
                            if (!mbar_wait(&full[stage], phase, abort_flag, status, spin)) { ok = false; break; }
                            tc_fence_after();
                        }
                        const uint32_t sa = smem_u32(stage_base + stage * STAGE_BYTES);
                        const uint32_t sa_lo = sa + A_BYTES;
                        const uint32_t sb_hi = sa + 2 * A_BYTES + s0 * SEG * 128;
                        const uint32_t sb_lo = sb_hi + B_BYTES;
#pragma unroll
                        for (int ks = 0; ks < BK / 8; ++ks) {
                            const uint32_t off = ks * 32;
                            const uint64_t dah = sdesc_sw128(sa + off), dal = sdesc_sw128(sa_lo + off);
                            const uint64_t dbh = sdesc_sw128(sb_hi + off), dbl = sdesc_sw128(sb_lo + off);
                            mma_tf32(d_main + col0, dah, dbh, idesc, ks == 0 ? fresh_main : 1u);
                            if (!early) {
                                mma_tf32(d_corr + col0, dah, dbl, idesc, ks == 0 ? fresh_corr : 1u);
                                mma_tf32(d_corr + col0, dal, dbh, idesc, 1);
                            }
                        }
                        mma_commit(&empty[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(main_full);
                    c0 = c1;
                }
            }
            mma_drain(drain_bar, status);   // every MMA issued has finished
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
            if (!warp_all(mbar_wait(&tq_full[qslot], qphase, abort_flag, status, spin))) break;
            const int t = ((volatile int*)tile_q)[qslot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tq_empty[qslot]);
            if (++qslot == QS) { qslot = 0; qphase ^= 1; }
            if (t < 0) break;
            const PTile& tl = tiles[t];
            const int l = tl.l, rt = tl.rt;
            const Steps sp = make_steps(dir, tl);
            const int row = rt * BM + quarter * 32 + lane;
            const int nch = min(max(tl.nseg - half * 4, 0), 4);   // my segments: half * 4 + ch
            const uint32_t tl_addr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.f;
            bool ok = true;
            for (int c0 = 0; c0 < sp.nsteps;) {
                const int c1 = sp.chunk_end(c0);
                if (!warp_all(mbar_wait(main_full, mphase, abort_flag, status, spin))) { ok = false; break; }
                mphase ^= 1;
                tc_fence_after();
                const bool last = c1 == sp.nsteps;
                c0 = c1;
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
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                if (ch >= nch) continue;
                const int s = half * 4 + ch;
                const BGroup G = groups[tl.g[s]];
                const int c = tl.c[s];
                const int nv = min(SEG, G.nl - c);   // valid lines of the segment
                const int N = G.N;
                const BTrans& T = trans[G.t];
                if (mode == kModeUserC64) {
                    float2* o = out_user + G.uoff + (size_t)(c >> 1) * N;
#pragma unroll
                    for (int j = 0; j < SEG; j += 2)
                        if (j < nv) o[(size_t)(j >> 1) * N + row] = make_float2(acc[ch * 32 + j], acc[ch * 32 + j + 1]);
                } else if (mode == kModePlanar) {
                    float* o = T.a_hi + (size_t)(G.bline0 + c) * N;
#pragma unroll
                    for (int j = 0; j < SEG; ++j)
                        if (j < nv) o[(size_t)j * N + row] = acc[ch * 32 + j];
                } else {
                    const float2 ph = T.phase[(size_t)(l & 1) * N + phase_entry(l, row, N)];
                    float* oh = T.b_hi + (size_t)(G.bline0 + c) * N;
                    float* ol = T.b_lo + (size_t)(G.bline0 + c) * N;
#pragma unroll
                    for (int j = 0; j < SEG; j += 2) {
                        if (j < nv) {
                            const float re = acc[ch * 32 + j] * ph.x - acc[ch * 32 + j + 1] * ph.y;
                            const float im = acc[ch * 32 + j] * ph.y + acc[ch * 32 + j + 1] * ph.x;
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

struct TileSet {
    PTile* d[2] = {nullptr, nullptr};   // forward, inverse
    int n[2] = {0, 0};
};

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
    dsbt::TMaps* tmaps_d = nullptr;
    dsbt::BMaps* cmaps_d = nullptr;
    std::vector<dsbt::BGroup> groups_h;
    dsbt::BGroup* groups_d = nullptr;
    dsbt::TileSet sets[dsbt::kOrders][3];  // tile lists per (order, width), built on demand
    int* sched = nullptr;
    int order = 3, ci = 2;                 // selected order and width index (autotuned)
    float tune_ms[dsbt::kOrders][3] = {{0}};
    std::vector<dsbt::GroupTable> gtab;   // per transform, for the sine/cosine kernels
    // interval scheme (DSBT_BATCH_INTERVAL): one DSBT_PLAN_FAST_SPLIT plan per
    // distinct grid, transforms spread over internal streams
    bool interval = false;
    std::vector<dsbt_plan*> fplans;        // per distinct grid (index cidx)
    std::vector<std::vector<int>> pcounts; // per distinct grid: channels of every l over its transforms
    std::vector<long long*> uoffs;         // per distinct grid: element offset of each merged channel
    std::vector<int> nchan_d;              // per distinct grid: merged channels
    std::vector<int> stream_of;            // per distinct grid
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;        // per stream, plus the fork event at the end
    std::vector<unsigned char*> sws;       // per stream workspace
    std::vector<size_t> sws_bytes;
};

namespace dsbt {
namespace {

void batch_free(dsbt_batch* b) {
    if (!b) return;
    for (auto* p : b->fplans) plan_release(p);
    for (auto* u : b->uoffs) cudaFree(u);
    for (auto* w : b->sws) cudaFree(w);
    for (auto e : b->joins) cudaEventDestroy(e);
    for (auto s_ : b->streams) cudaStreamDestroy(s_);
    if (b->shared) plan_release(b->shared);
    for (auto* p : b->tw) plan_release(p);
    cudaFree(b->comp);
    cudaFree(b->comp64);
    cudaFree(b->ws);
    cudaFree(b->trans_d);
    cudaFree(b->tmaps_d);
    cudaFree(b->cmaps_d);
    cudaFree(b->groups_d);
    for (auto& row : b->sets)
        for (auto& ts : row) {
            cudaFree(ts.d[0]);
            cudaFree(ts.d[1]);
        }
    cudaFree(b->sched);
    delete b;
}

const int kBnCaps[3] = {128, 192, 256};

// (transform, l) groups with at least one channel, transform-major.
std::vector<BGroup> make_groups(const dsbt_batch* b) {
    std::vector<BGroup> gs;
    for (int t = 0; t < b->T; ++t) {
        const int off = b->counts_off[t];
        int chan = 0;
        for (int l = 0; l <= b->lmax[t]; ++l) {
            const int c = b->counts[off + l];
            if (c > 0) {
                BGroup G;
                G.t = t;
                G.l = l;
                G.N = b->N[t];
                G.nl = 2 * c;
                G.bline0 = 2 * chan;
                G.cidx = b->cidx[t];
                G.uoff = b->uoff[t] + (long long)chan * G.N;
                gs.push_back(G);
            }
            chan += c;
        }
    }
    return gs;
}

// Packs the segments of a list of groups, in order, into tiles of at most
// segcap segments at row tile rt of l.  A forward tile's K range is that of
// its smallest grid (all grids hold rows up to (rt + 1) BM); an inverse tile's
// is that of its first, largest grid, and its classes are the runs of equal N.
struct TileBuilder {
    std::vector<PTile> out;
    int segcap = SEG_MAX;
    int dir = 1;
    void push(PTile& cur, const std::vector<BGroup>& gs) {
        if (!cur.nseg) return;
        cur.ncls = 0;
        for (int s = 0; s < cur.nseg; ++s) {
            const BGroup& G = gs[cur.g[s]];
            if (dir > 0) {
                if (s == 0 || G.N < cur.N) { cur.N = G.N; cur.cidx = G.cidx; }
            } else if (s == 0) {
                cur.N = G.N;
                cur.cidx = G.cidx;
            }
            const bool new_class = dir < 0 && s > 0 && G.N != gs[cur.g[s - 1]].N;
            if (new_class) cur.cend[cur.ncls++] = (unsigned char)s;
        }
        cur.cend[cur.ncls++] = (unsigned char)cur.nseg;
        out.push_back(cur);
        memset(&cur, 0, sizeof(cur));
    }
    void add(const std::vector<BGroup>& gs, const std::vector<int>& gi, int l, int rt) {
        PTile cur;
        memset(&cur, 0, sizeof(cur));
        for (int g : gi)
            for (int c = 0; c < gs[g].nl; c += SEG) {
                if (cur.nseg == segcap) push(cur, gs);
                cur.l = l;
                cur.rt = rt;
                cur.g[cur.nseg] = g;
                cur.c[cur.nseg] = c;
                ++cur.nseg;
            }
        push(cur, gs);
    }
};

// Tile list of one direction (dir > 0 forward).  Orders: 0 transform-major
// (largest transform first, l descending), 1 l-major (l descending, N
// descending), both with each group's tiles together; 2 l-major with row tiles
// interleaved across the transforms of one l, so tiles reading the same slab of
// the shared factors run together; 3 as 2 with segments of different transforms
// packed into one tile.  Forward row tiles run longest K first with rt = 0 last
// (orders 2, 3) or first (orders 0, 1); inverse row tiles ascending.
std::vector<PTile> make_tiles(const dsbt_batch* b, const std::vector<BGroup>& gs, int order, int segcap, int dir) {
    std::vector<int> idx(gs.size());
    for (size_t i = 0; i < gs.size(); ++i) idx[i] = (int)i;
    if (order == 0) {
        std::vector<double> tw(b->T, 0.0);
        for (const BGroup& G : gs) tw[G.t] += (double)G.nl * G.N * G.N;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            const BGroup &X = gs[x], &Y = gs[y];
            if (X.t != Y.t) return tw[X.t] > tw[Y.t] || (tw[X.t] == tw[Y.t] && X.t < Y.t);
            return X.l > Y.l;
        });
    } else {
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) {
            const BGroup &X = gs[x], &Y = gs[y];
            if (X.l != Y.l) return X.l > Y.l;
            return X.N > Y.N;
        });
    }
    TileBuilder tb;
    tb.segcap = segcap;
    tb.dir = dir;
    if (order <= 1) {
        for (int g : idx) {
            const int RT = gs[g].N / BM;
            for (int q = 0; q < RT; ++q) {
                const int rt = (dir > 0) ? (q == 0 ? 0 : RT - q) : q;
                tb.add(gs, {g}, gs[g].l, rt);
            }
        }
        return tb.out;
    }
    size_t i = 0;
    while (i < idx.size()) {
        const int l = gs[idx[i]].l;
        size_t j = i;
        while (j < idx.size() && gs[idx[j]].l == l) ++j;
        const int rtmax = gs[idx[i]].N / BM;   // N descending inside the block
        std::vector<int> rts;
        if (dir > 0) {
            for (int rt = rtmax - 1; rt >= 1; --rt) rts.push_back(rt);
            rts.push_back(0);
        } else {
            for (int rt = 0; rt < rtmax; ++rt) rts.push_back(rt);
        }
        for (int rt : rts) {
            if (order == 2) {
                for (size_t k = i; k < j; ++k)
                    if (rt < gs[idx[k]].N / BM) tb.add(gs, {idx[k]}, l, rt);
            } else if (dir < 0 || rt >= 1) {   // pack all grids that hold row tile rt
                std::vector<int> gi;
                for (size_t k = i; k < j; ++k)
                    if (rt < gs[idx[k]].N / BM) gi.push_back(idx[k]);
                tb.add(gs, gi, l, rt);
            } else {                           // forward rt = 0 reads per-N rows: one grid per tile
                size_t k = i;
                while (k < j) {
                    const int N = gs[idx[k]].N;
                    std::vector<int> gi;
                    while (k < j && gs[idx[k]].N == N) gi.push_back(idx[k++]);
                    tb.add(gs, gi, l, rt);
                }
            }
        }
        i = j;
    }
    return tb.out;
}

// Host check of a tile list against the rules the kernel relies on.
bool tiles_valid(const std::vector<BGroup>& gs, const std::vector<PTile>& ts, int dir) {
    for (const PTile& p : ts) {
        if (p.nseg < 1 || p.nseg > SEG_MAX || p.ncls < 1 || p.ncls > p.nseg || p.cend[p.ncls - 1] != p.nseg)
            return false;
        int cls = 0;
        for (int s = 0; s < p.nseg; ++s) {
            const BGroup& G = gs[p.g[s]];
            if (G.l != p.l || p.c[s] < 0 || p.c[s] >= G.nl || p.c[s] % SEG) return false;
            if (p.rt >= G.N / BM) return false;   // every output row exists in the segment's grid
            if (s == p.cend[cls]) ++cls;
            const BGroup& F = gs[p.g[cls == 0 ? 0 : p.cend[cls - 1]]];   // first segment of the class
            if (dir < 0 && (G.N != F.N || G.cidx != F.cidx)) return false;
            if (dir > 0) {
                if (G.N < p.N || (p.rt == 0 && (G.N != p.N || G.cidx != p.cidx))) return false;
            } else {
                if (G.N > p.N || (cls > 0 && G.N >= gs[p.g[p.cend[cls - 1] - 1]].N)) return false;
            }
        }
        if (dir > 0 && p.ncls != 1) return false;
    }
    return true;
}

// Builds (once) the forward and inverse tile lists of one (order, width)
// variant.  Lists are immutable once built, so graphs captured with one stay
// valid when another variant is selected.
int ensure_tiles(dsbt_batch* b, int order, int ci, cudaStream_t st) {
    TileSet& ts = b->sets[order][ci];
    if (ts.d[0]) return DSBT_OK;
    for (int d = 0; d < 2; ++d) {
        const int dir = d == 0 ? +1 : -1;
        std::vector<PTile> tl = make_tiles(b, b->groups_h, order, kBnCaps[ci] / SEG, dir);
        if (!tiles_valid(b->groups_h, tl, dir)) {
            set_error("internal error: invalid tile list (order %d, width %d)", order, kBnCaps[ci]);
            return DSBT_ERR_INVALID;
        }
        ts.n[d] = (int)tl.size();
        if (cudaMalloc((void**)&ts.d[d], std::max<size_t>(1, tl.size()) * sizeof(PTile)) != cudaSuccess) {
            cudaGetLastError();
            set_error("tile list allocation failed");
            return DSBT_ERR_NOMEM;
        }
        DSBT_CUDA_TRY(cudaMemcpyAsync(ts.d[d], tl.data(), tl.size() * sizeof(PTile), cudaMemcpyHostToDevice, st));
    }
    DSBT_CUDA_TRY(cudaStreamSynchronize(st));
    return DSBT_OK;
}

void free_tiles(TileSet& ts) {
    cudaFree(ts.d[0]);
    cudaFree(ts.d[1]);
    ts.d[0] = ts.d[1] = nullptr;
    ts.n[0] = ts.n[1] = 0;
}

int launch_contract(const dsbt_batch* b, int order, int ci, int dir, int mode, float2* out_user, cudaStream_t st) {
    const TileSet& ts = b->sets[order][ci];
    const int d = dir > 0 ? 0 : 1;
    const int total = ts.n[d];
    if (!ts.d[d]) {
        set_error("internal error: tile list not built");
        return DSBT_ERR_INVALID;
    }
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    if (int rc0 = ensure_smem((const void*)k_contract_batch, smem)) return rc0;
    int dev = 0, nsm = 0;
    DSBT_CUDA_TRY(cudaGetDevice(&dev));
    DSBT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = total < nsm ? total : nsm;
    if (grid == 0) return DSBT_OK;
    DSBT_CUDA_TRY(cudaMemsetAsync(b->sched, 0, sizeof(int), st));
    const dsbt_plan* s = b->shared;
    ProfScope ps(kKContractTF32, st);
    k_contract_batch<<<grid, NTHREADS, smem, st>>>(s->tm_T_hi, s->tm_T_lo, b->tF96_hi, b->tF96_lo, s->tm_Tt_hi,
                                                   s->tm_Tt_lo, ts.d[d], total, b->groups_d, b->trans_d, b->tmaps_d,
                                                   b->cmaps_d, b->Nmax, dir, mode, out_user, s->status, s->spin_limit,
                                                   b->sched);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

// Interval scheme: the transforms of each distinct grid form one grouped call
// on that grid's plan (channels of every l gathered from the batch array
// through the grid's offset table), in the batch's internal streams (forked
// from and joined back into st, so a capture of st takes the whole fork-join
// graph).
int run_batch_interval(const dsbt_batch* b, int kinetic, double tau, const float* in, float* out, cudaStream_t st) {
    const int S = (int)b->streams.size();
    cudaEvent_t fork = b->joins[S];
    DSBT_CUDA_TRY(cudaEventRecord(fork, st));
    for (int k = 0; k < S; ++k) DSBT_CUDA_TRY(cudaStreamWaitEvent(b->streams[k], fork, 0));
    for (size_t d = 0; d < b->fplans.size(); ++d) {
        if (b->nchan_d[d] == 0) continue;
        const int k = b->stream_of[d];
        const int rc = grouped_device_call(kinetic ? 2 : 0, b->fplans[d], b->pcounts[d].data(), DSBT_C64, tau, in, out,
                                           b->sws[k], b->sws_bytes[k], b->streams[k], b->uoffs[d]);
        if (rc) return rc;
    }
    for (int k = 0; k < S; ++k) {
        DSBT_CUDA_TRY(cudaEventRecord(b->joins[k], b->streams[k]));
        DSBT_CUDA_TRY(cudaStreamWaitEvent(st, b->joins[k], 0));
    }
    return DSBT_OK;
}

int run_batch(const dsbt_batch* b, int kinetic, double tau, const float* in, float* out, cudaStream_t st) {
    if (b->interval) return run_batch_interval(b, kinetic, tau, in, out, st);
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
    if (!kinetic) return launch_contract(b, b->order, b->ci, +1, kModeUserC64, (float2*)out, st);
    rc = launch_contract(b, b->order, b->ci, +1, kModeSplit, nullptr, st);
    if (!rc) rc = launch_contract(b, b->order, b->ci, -1, kModePlanar, nullptr, st);
    if (rc) return rc;
    for (int t = 0; t < b->T; ++t) {
        const dsbt_plan* tp = b->tw[b->cidx[t]];
        rc = dct_inverse_f32(tp, b->gtab[t], true, b->trans_h[t].a_hi, out + 2 * b->uoff[t], st);
        if (rc) return rc;
    }
    return DSBT_OK;
}

// Times the forward contraction for each (order, column-tile width) on the
// batch's own shapes (workspace contents do not affect the timing), keeps the
// fastest and frees the other tile lists (no graph can hold them yet).
int autotune(dsbt_batch* b, cudaStream_t st) {
    cudaEvent_t e0, e1;
    DSBT_CUDA_TRY(cudaEventCreate(&e0));
    DSBT_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int rc = DSBT_OK;
    for (int order = 0; order < kOrders && !rc; ++order) {
        for (int ci = 0; ci < 3 && !rc; ++ci) {
            rc = ensure_tiles(b, order, ci, st);
            if (!rc) rc = launch_contract(b, order, ci, +1, kModeSplit, nullptr, st);   // warm-up
            if (rc) break;
            DSBT_CUDA_TRY(cudaEventRecord(e0, st));
            rc = launch_contract(b, order, ci, +1, kModeSplit, nullptr, st);
            if (rc) break;
            DSBT_CUDA_TRY(cudaEventRecord(e1, st));
            DSBT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            DSBT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            b->tune_ms[order][ci] = ms;
            if (ms < best) {
                best = ms;
                b->order = order;
                b->ci = ci;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    for (int order = 0; order < kOrders; ++order)
        for (int ci = 0; ci < 3; ++ci)
            if (order != b->order || ci != b->ci) free_tiles(b->sets[order][ci]);
    return DSBT_OK;
}

}  // namespace
}  // namespace dsbt

using namespace dsbt;

namespace dsbt {
namespace {

// Host-side description of a batch (sizes, offsets, distinct grids); touches
// no device memory.
int batch_describe(dsbt_batch* b, int ntrans, const int* N, const int* l_max, const int* counts, double dr) {
    DSBT_CHECK_ARG(N != nullptr && l_max != nullptr && counts != nullptr, "dsbt_batch: NULL argument");
    DSBT_CHECK_ARG(ntrans >= 1 && ntrans <= 4096, "dsbt_batch: ntrans=%d out of range", ntrans);
    DSBT_CHECK_ARG(dr > 0.0 && isfinite(dr), "dsbt_batch: dr must be positive");
    b->T = ntrans;
    b->dr = dr;
    int off = 0;
    long long uoff = 0;
    for (int t = 0; t < ntrans; ++t) {
        DSBT_CHECK_ARG(N[t] >= 256 && N[t] <= 8192 && N[t] % 256 == 0 && l_max[t] >= 0 && l_max[t] <= 64,
                       "dsbt_batch: transform %d: N=%d, l_max=%d not supported", t, N[t], l_max[t]);
        b->N.push_back(N[t]);
        b->lmax.push_back(l_max[t]);
        b->counts_off.push_back(off);
        int nc = 0;
        for (int l = 0; l <= l_max[t]; ++l) {
            DSBT_CHECK_ARG(counts[off + l] >= 0 && counts[off + l] <= (1 << 24), "dsbt_batch: bad channel count");
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
        auto it = std::find(b->dN.begin(), b->dN.end(), N[t]);
        if (it == b->dN.end()) {
            b->cidx.push_back((int)b->dN.size());
            b->dN.push_back(N[t]);
        } else {
            b->cidx.push_back((int)(it - b->dN.begin()));
        }
    }
    b->total_elems = uoff;
    b->groups_h = make_groups(b);
    return DSBT_OK;
}

}  // namespace
}  // namespace dsbt

extern "C" int dsbt_batch_tiles(int ntrans, const int* N, const int* l_max, const int* counts, int order,
                                int bn_cap, int* ntiles_fwd, int* ntiles_inv, long long* seg_lines) {
    DSBT_CHECK_ARG(order >= 0 && order < kOrders, "dsbt_batch_tiles: order %d not in 0..%d", order, kOrders - 1);
    DSBT_CHECK_ARG(bn_cap == 128 || bn_cap == 192 || bn_cap == 256, "dsbt_batch_tiles: width %d", bn_cap);
    dsbt_batch tmp;
    int rc = batch_describe(&tmp, ntrans, N, l_max, counts, 1.0);
    if (rc) return rc;
    long long lines = 0;
    for (int d = 0; d < 2; ++d) {
        const int dir = d == 0 ? +1 : -1;
        std::vector<PTile> tl = make_tiles(&tmp, tmp.groups_h, order, bn_cap / SEG, dir);
        if (!tiles_valid(tmp.groups_h, tl, dir)) {
            set_error("dsbt_batch_tiles: invalid tile list (order %d, width %d, dir %d)", order, bn_cap, dir);
            return DSBT_ERR_INVALID;
        }
        if (d == 0 && ntiles_fwd) *ntiles_fwd = (int)tl.size();
        if (d == 1 && ntiles_inv) *ntiles_inv = (int)tl.size();
        if (d == 0)
            for (const PTile& p : tl) lines += (long long)p.nseg * SEG;
    }
    if (seg_lines) *seg_lines = lines;
    return DSBT_OK;
}

namespace dsbt {
namespace {

// The interval-scheme batch: plans per distinct grid, streams, workspaces.
int create_interval(dsbt_batch* b, cudaStream_t st) {
    b->interval = true;
    const int ND = (int)b->dN.size();
    std::vector<int> lmax_d(ND, 0);
    for (int t = 0; t < b->T; ++t) lmax_d[b->cidx[t]] = std::max(lmax_d[b->cidx[t]], b->lmax[t]);
    for (int d = 0; d < ND; ++d) {
        dsbt_plan* p = nullptr;
        const int rc = dsbt_plan_create(b->dN[d], b->dN[d] * b->dr, lmax_d[d], DSBT_PLAN_FAST_SPLIT, st, &p);
        if (rc) return rc;
        b->fplans.push_back(p);
    }
    // merged calls: per grid, the channels of every l over its transforms in
    // batch order, with their element offsets in the batch array
    b->pcounts.assign(ND, {});
    b->nchan_d.assign(ND, 0);
    std::vector<std::vector<long long>> offs(ND);
    for (int d = 0; d < ND; ++d) {
        b->pcounts[d].assign(lmax_d[d] + 1, 0);
        for (int l = 0; l <= lmax_d[d]; ++l)
            for (int t = 0; t < b->T; ++t) {
                if (b->cidx[t] != d || l > b->lmax[t]) continue;
                int c0 = 0;
                for (int q = 0; q < l; ++q) c0 += b->counts[b->counts_off[t] + q];
                const int c = b->counts[b->counts_off[t] + l];
                for (int i = 0; i < c; ++i) offs[d].push_back(b->uoff[t] + (long long)(c0 + i) * b->dN[d]);
                b->pcounts[d][l] += c;
            }
        b->nchan_d[d] = (int)offs[d].size();
        long long* u = nullptr;
        if (!offs[d].empty()) {
            if (cudaMalloc((void**)&u, offs[d].size() * sizeof(long long)) != cudaSuccess ||
                cudaMemcpy(u, offs[d].data(), offs[d].size() * sizeof(long long), cudaMemcpyHostToDevice) !=
                    cudaSuccess) {
                cudaGetLastError();
                cudaFree(u);
                set_error("dsbt_batch_create: offset table upload failed");
                return DSBT_ERR_NOMEM;
            }
        }
        b->uoffs.push_back(u);
    }
    // grids by decreasing work, each to the least loaded stream
    const int S = std::min(4, ND);
    std::vector<int> ord(ND);
    for (int d = 0; d < ND; ++d) ord[d] = d;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
        return (double)b->dN[x] * b->nchan_d[x] > (double)b->dN[y] * b->nchan_d[y];
    });
    std::vector<double> load(S, 0.0);
    std::vector<size_t> need(S, 0);
    b->stream_of.assign(ND, 0);
    for (int d : ord) {
        const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->stream_of[d] = k;
        load[k] += (double)b->dN[d] * b->nchan_d[d];
        need[k] = std::max(need[k], dsbt_workspace_size(b->fplans[d], b->nchan_d[d], DSBT_C64));
    }
    for (int k = 0; k < S; ++k) {
        cudaStream_t sk = nullptr;
        DSBT_CUDA_TRY(cudaStreamCreateWithFlags(&sk, cudaStreamNonBlocking));
        b->streams.push_back(sk);
        unsigned char* w = nullptr;
        if (cudaMalloc((void**)&w, need[k] + 256) != cudaSuccess) {
            cudaGetLastError();
            set_error("dsbt_batch_create: workspace allocation of %zu bytes failed", need[k]);
            return DSBT_ERR_NOMEM;
        }
        b->sws.push_back(w);
        b->sws_bytes.push_back(need[k] + 256);
    }
    for (int k = 0; k <= S; ++k) {
        cudaEvent_t e = nullptr;
        DSBT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->joins.push_back(e);
    }
    DSBT_CUDA_TRY(cudaStreamSynchronize(st));
    return DSBT_OK;
}

}  // namespace
}  // namespace dsbt

extern "C" int dsbt_batch_create(int ntrans, const int* N, const int* l_max, const int* counts, double dr,
                                 int autotune_tiles, void* stream, dsbt_batch** out) {
    return dsbt_batch_create_ex(ntrans, N, l_max, counts, dr, autotune_tiles ? DSBT_BATCH_AUTOTUNE : 0, stream, out);
}

extern "C" int dsbt_batch_create_ex(int ntrans, const int* N, const int* l_max, const int* counts, double dr,
                                    int flags, void* stream, dsbt_batch** out) {
    DSBT_CHECK_ARG(out != nullptr, "dsbt_batch_create: NULL argument");
    DSBT_CHECK_ARG((flags & ~(DSBT_BATCH_AUTOTUNE | DSBT_BATCH_INTERVAL)) == 0, "dsbt_batch_create: flags=%d invalid",
                   flags);
    *out = nullptr;
    const int autotune_tiles = (flags & DSBT_BATCH_AUTOTUNE) != 0;
    cudaStream_t st = (cudaStream_t)stream;
    dsbt_batch* b = new (std::nothrow) dsbt_batch();
    if (!b) return DSBT_ERR_NOMEM;
    {
        const int rc0 = batch_describe(b, ntrans, N, l_max, counts, dr);
        if (rc0) { delete b; return rc0; }
    }
    if (flags & DSBT_BATCH_INTERVAL) {
        const int rc1 = create_interval(b, st);
        if (rc1) { batch_free(b); return rc1; }
        *out = b;
        return DSBT_OK;
    }
    // shared factors at (N_max, l_max)
    int rc = dsbt_plan_create(b->Nmax, b->Nmax * dr, b->L - 1, DSBT_PLAN_TF32X3, stream, &b->shared);
    if (rc) { batch_free(b); return rc; }
    rc = encode_tmap_f32_sw128(&b->tF96_hi, b->shared->Thi, (uint64_t)b->L * b->Nmax, b->Nmax, 96, 32);
    if (!rc) rc = encode_tmap_f32_sw128(&b->tF96_lo, b->shared->Tlo, (uint64_t)b->L * b->Nmax, b->Nmax, 96, 32);
    if (rc) { batch_free(b); return rc; }
    // distinct grids: twiddles and per-N tables
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
    std::vector<TMaps> tm(ntrans);
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
        for (int k = 0; k < 3 && !rc; ++k) {
            const int box = SEG << k;
            rc = encode_tmap_f32_sw128(&tm[t].m[4 * k + 0], T.a_hi, rows, N[t], box, 32);
            if (!rc) rc = encode_tmap_f32_sw128(&tm[t].m[4 * k + 1], T.a_lo, rows, N[t], box, 32);
            if (!rc) rc = encode_tmap_f32_sw128(&tm[t].m[4 * k + 2], T.b_hi, rows, N[t], box, 32);
            if (!rc) rc = encode_tmap_f32_sw128(&tm[t].m[4 * k + 3], T.b_lo, rows, N[t], box, 32);
        }
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
              cudaMalloc((void**)&b->tmaps_d, ntrans * sizeof(TMaps)) == cudaSuccess &&
              cudaMalloc((void**)&b->cmaps_d, ND * sizeof(BMaps)) == cudaSuccess;
    ok = ok && cudaMemcpy(b->trans_d, b->trans_h.data(), ntrans * sizeof(BTrans), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->tmaps_d, tm.data(), ntrans * sizeof(TMaps), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(b->cmaps_d, cm.data(), ND * sizeof(BMaps), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        batch_free(b);
        set_error("dsbt_batch_create: table upload failed");
        return DSBT_ERR_CUDA;
    }
    if (!b->groups_h.empty()) {
        const size_t gb = b->groups_h.size() * sizeof(BGroup);
        if (cudaMalloc((void**)&b->groups_d, gb) != cudaSuccess ||
            cudaMemcpy(b->groups_d, b->groups_h.data(), gb, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            batch_free(b);
            set_error("dsbt_batch_create: group table upload failed");
            return DSBT_ERR_CUDA;
        }
    }
    rc = ensure_tiles(b, b->order, b->ci, st);
    if (rc) { batch_free(b); return rc; }
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
    if (order) *order = b->interval ? -1 : b->order;
    if (bn_cap) *bn_cap = b->interval ? 0 : kBnCaps[b->ci];
    if (tune_ms)
        for (int o = 0; o < kOrders; ++o)
            for (int c = 0; c < 3; ++c) tune_ms[o * 3 + c] = b->tune_ms[o][c];
    return DSBT_OK;
}

extern "C" int dsbt_batch_set_tiles(dsbt_batch* b, int order, int bn_cap, void* stream) {
    DSBT_CHECK_ARG(b != nullptr, "dsbt_batch_set_tiles: NULL batch");
    if (b->interval) {
        set_error("dsbt_batch_set_tiles: a batch on the interval scheme has no tile list");
        return DSBT_ERR_UNSUPPORTED;
    }
    DSBT_CHECK_ARG(order >= 0 && order < kOrders, "dsbt_batch_set_tiles: order %d not in 0..%d", order, kOrders - 1);
    int ci = -1;
    for (int c = 0; c < 3; ++c)
        if (kBnCaps[c] == bn_cap) ci = c;
    DSBT_CHECK_ARG(ci >= 0, "dsbt_batch_set_tiles: width %d not 128, 192 or 256", bn_cap);
    const int rc = ensure_tiles(b, order, ci, (cudaStream_t)stream);
    if (rc) return rc;
    b->order = order;
    b->ci = ci;
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
