// gemm_tf32x3.cu -- compensated split-TF32 contraction with T_l on the sm_103a
// tensor cores (tcgen05 + TMA + TMEM).
//
// Forward (Eq. (24)):  b[c][n] = sum_m T_l[n][m] f[c][m]     A = T_l
// Inverse (Eq. (25)):  f[c][m] = sum_n T_l[n][m] b[c][n]     A = T_l^T
// Both operands are split into TF32 pairs, X = X_hi + X_lo, and each K step
// issues three MMAs into FP32 TMEM accumulators:
//     D_main += A_hi B_hi,   D_corr += A_hi B_lo + A_lo B_hi
// (A_lo B_lo ~ 2^-22 dropped), which keeps about 2^-21 relative accuracy per
// product while every MMA runs at TF32 tensor rate.
//
// Tiles: 128 output rows (TMEM lanes) x up to 256 real lines (TMEM columns);
// K in blocks of 32 (one 128-byte swizzle row of FP32).  A tile never reads the
// zero upper triangle of T_l: forward row tile [r0, r0+128) reads K < r0+128
// (all K when it holds completion rows); inverse tile reads the completion rows
// (K < n_extra <= 32) and K >= r0.
//
// CTA roles (320 threads, one CTA per SM, persistent over a cost-ordered tile
// list): warp 0 = TMA producer, warp 1 = TMEM owner + MMA issuer, warps 2-9 =
// epilogue (two warps per TMEM lane quarter, 128 columns each: drain the main
// accumulator every KC K-blocks into FP32 registers, then the optional kinetic
// phase + TF32 split, then global stores, which overlap the next tile's MMAs).
// Every mbarrier wait is bounded: on expiry the kernel records kStatusTimeout
// in the plan's status word and all roles leave their loops.
#include "plan.cuh"
#include "tc_ptx.cuh"

namespace dsbt {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BK = 32;
constexpr int BN_MAX = 256;
constexpr int BBOX = 64;                           // rows per B TMA box
constexpr int STAGES = 2;
constexpr int KC = 4;                              // K blocks per main-accumulator chunk
constexpr int EPI_WARPS = 8;
constexpr int QS = 4;                              // tile-queue slots (scheduler -> MMA, epilogue)
constexpr int A_BYTES = BM * BK * 4;               // 16 KiB
constexpr int B_BYTES = BN_MAX * BK * 4;           // 32 KiB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
// B lines are re-read by every row tile of their group: keep them in L2.
#ifndef DSBT_B_EVICT_LAST
#define DSBT_B_EVICT_LAST 1
#endif

// Tiles are visited group by group, largest l first (the groups with the most
// work), and inside a group by cost level (row tiles with the longest K range
// first), then column tile.  Consecutive tiles then share a row slab of T_l in
// L2, and a group's B lines (<= 67 MB at the largest configuration) stay in L2
// while all its row tiles use them.
struct TileSpace {
    int RT;                        // row tiles (N / 128)
    int KB;                        // K blocks (N / 32)
    int total;                     // sum over groups of RT * CT
    int order[kMaxGroups];         // group visited at position i
    int t0[kMaxGroups + 1];        // first tile of position i
    int ct[kMaxGroups];            // column tiles of the group at position i
};

// ------------------------------------------------------------ tile decode

struct Tile {
    int g, rt, ct, nmma;
};

__device__ __forceinline__ Tile decode(const TileSpace& ts, const GroupTable& gt, int dir, int t) {
    Tile tl;
    int i = 0;
    while (ts.t0[i + 1] <= t) ++i;
    const int g = ts.order[i];
    const int local = t - ts.t0[i];
    const int q = local / ts.ct[i];
    tl.g = g;
    tl.ct = local - q * ts.ct[i];
    tl.rt = (dir > 0) ? (q == 0 ? 0 : ts.RT - q) : q;
    const int nl = gt.line0[g + 1] - gt.line0[g];
    int left = nl - tl.ct * BN_MAX;
    if (left > BN_MAX) left = BN_MAX;
    tl.nmma = (left + 15) & ~15;
    return tl;
}

// K blocks of an output row tile, as two half-open ranges [a0, a1) and
// [b0, b1) (b empty unless the inverse reads completion rows and a diagonal
// band).  Forward tiles walk K upwards from 0 and inverse tiles walk it
// downwards from N, so every tile of a group starts at the same K block and the
// tiles running at the same time stream the same B blocks through L2.
struct KRange {
    int a0, a1, b0, b1, up;
    __device__ __forceinline__ int count() const { return (a1 - a0) + (b1 - b0); }
    // i-th block in walking order
    __device__ __forceinline__ int at(int i) const {
        if (up) return (i < a1 - a0) ? (a0 + i) : (b0 + i - (a1 - a0));
        const int nb = b1 - b0;
        return (i < nb) ? (b1 - 1 - i) : (a1 - 1 - (i - nb));
    }
};

__device__ __forceinline__ KRange kranges(int dir, int rt, int nx, int KB) {
    KRange k;
    const int r0 = rt * BM;
    k.up = dir > 0;
    k.a0 = 0;
    k.b0 = k.b1 = 0;
    if (r0 < nx) { k.a1 = KB; return k; }
    if (dir > 0) { k.a1 = min(KB, (r0 + BM) / BK); return k; }
    k.a1 = (nx + BK - 1) / BK;
    k.b0 = max(k.a1, r0 / BK);
    k.b1 = KB;
    return k;
}

// ------------------------------------------------------------ the kernel

struct EpiArgs {
    int mode;              // OutMode
    float* out0;
    float* out1;
    const float2* phase;   // [2][N] by parity of l, [l_max+1][N] when per_l, or nullptr
    int per_l;
};

// TMEM layout (512 columns): [0, 256) main accumulator A_hi B_hi of the
// current K chunk; [256, 512) correction accumulator A_hi B_lo + A_lo B_hi of
// the whole tile.  The tensor cores accumulate with truncation, so the main
// sum is restarted every KC blocks and the chunk sums are added in FP32 with
// round-to-nearest in the epilogue's registers; the correction terms are
// 2^-11 smaller and stay in TMEM for the whole tile.
__global__ void __launch_bounds__(NTHREADS, 1)
k_contract_tf32x3(const __grid_constant__ CUtensorMap tmA_hi, const __grid_constant__ CUtensorMap tmA_lo,
                  const __grid_constant__ CUtensorMap tmB_hi, const __grid_constant__ CUtensorMap tmB_lo,
                  GroupTable gt, TileSpace ts, int N, int dir, EpiArgs ep, unsigned* status,
                  uint32_t spin, int* sched) {
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
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            StageLedger led;
#if DSBT_B_EVICT_LAST
            const uint64_t pol_b = policy_evict_last();
#endif
            int qslot = 0;
            uint32_t qphase = 0;
            while (ok) {
                // dynamic tile scheduler: the next tile of the ordered list goes to
                // whichever CTA asks first, so the tiles in flight always form one
                // contiguous window of the list (at most two groups' B lines live in L2)
                if (!mbar_wait(&tq_empty[qslot], qphase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                int t = atomicAdd(sched, 1);
                if (t >= ts.total) t = -1;
                tile_q[qslot] = t;
                mbar_arrive(&tq_full[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (t < 0) break;
                const Tile tl = decode(ts, gt, dir, t);
                const int l = gt.l[tl.g];
                const KRange kr = kranges(dir, tl.rt, n_extra(l), ts.KB);
                const int nbox = (tl.nmma + BBOX - 1) / BBOX;
                const uint32_t bytes = 2 * A_BYTES + 2 * nbox * BBOX * BK * 4;
                const int arow = l * N + tl.rt * BM;
                const int brow = gt.line0[tl.g] + tl.ct * BN_MAX;
                const int nkb = kr.count();
                for (int i = 0; i < nkb; ++i) {
                    const int kb = kr.at(i);
                    if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                    unsigned char* sb = stage_base + stage * STAGE_BYTES;
                    mbar_expect_tx(&full[stage], bytes);
                    led.arm(stage, phase);
                    tma_load_2d(sb, &tmA_hi, &full[stage], kb * BK, arow);
                    tma_load_2d(sb + A_BYTES, &tmA_lo, &full[stage], kb * BK, arow);
                    for (int b = 0; b < nbox; ++b) {
#if DSBT_B_EVICT_LAST
                        tma_load_2d_hint(sb + 2 * A_BYTES + b * BBOX * 128, &tmB_hi, &full[stage], kb * BK,
                                         brow + b * BBOX, pol_b);
                        tma_load_2d_hint(sb + 2 * A_BYTES + B_BYTES + b * BBOX * 128, &tmB_lo, &full[stage],
                                         kb * BK, brow + b * BBOX, pol_b);
#else
                        tma_load_2d(sb + 2 * A_BYTES + b * BBOX * 128, &tmB_hi, &full[stage], kb * BK,
                                    brow + b * BBOX);
                        tma_load_2d(sb + 2 * A_BYTES + B_BYTES + b * BBOX * 128, &tmB_lo, &full[stage],
                                    kb * BK, brow + b * BBOX);
#endif
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
                const Tile tl = decode(ts, gt, dir, t);
                const int l = gt.l[tl.g];
                const KRange kr = kranges(dir, tl.rt, n_extra(l), ts.KB);
                const uint32_t idesc = idesc_tf32(BM, tl.nmma);
                const int nkb = kr.count();
                uint32_t acc_corr = 0;
                for (int c0 = 0; c0 < nkb && ok; c0 += KC) {
                    const int c1 = min(nkb, c0 + KC);
                    // Inside a tile, the first K block's correction products (which do
                    // not touch the main accumulator) go out before the wait for the
                    // epilogue to drain the main accumulator, keeping the tensor pipe
                    // busy during the drain.  At a tile start the epilogue may still be
                    // reading the previous tile's correction sum, so nothing goes early.
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
                            mma_tf32(d_corr, dah, dbl, idesc, 1);
                            mma_tf32(d_corr, dal, dbh, idesc, 1);
                        }
                    }
                    // the epilogue must have drained the previous chunk (and, at a
                    // tile start, read the previous tile's correction sum)
                    if (!mbar_wait(main_empty, mphase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                    mphase ^= 1;
                    tc_fence_after();
                    uint32_t acc_main = 0;
                    for (int i = c0; i < c1; ++i) {
                        const bool early = pre && i == c0;   // correction products already issued
                        if (!early) {
                            if (!mbar_wait(&full[stage], phase, abort_flag, status, spin)) { ok = false; break; }
                            tc_fence_after();
                        }
                        const uint32_t sa = smem_u32(stage_base + stage * STAGE_BYTES);
                        const uint32_t sa_lo = sa + A_BYTES;
                        const uint32_t sb_hi = sa + 2 * A_BYTES;
                        const uint32_t sb_lo = sb_hi + B_BYTES;
#pragma unroll
                        for (int ks = 0; ks < BK / 8; ++ks) {
                            const uint32_t off = ks * 32;   // 8 TF32 values = 32 bytes along K
                            const uint64_t dah = sdesc_sw128(sa + off), dal = sdesc_sw128(sa_lo + off);
                            const uint64_t dbh = sdesc_sw128(sb_hi + off), dbl = sdesc_sw128(sb_lo + off);
                            mma_tf32(d_main, dah, dbh, idesc, acc_main);
                            if (!early) {
                                mma_tf32(d_corr, dah, dbl, idesc, acc_corr);
                                mma_tf32(d_corr, dal, dbh, idesc, 1);
                            }
                            acc_main = 1;
                            acc_corr = 1;
                        }
                        mma_commit(&empty[stage]);   // frees the stage once these MMAs finish
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(main_full);
                }
            }
            mma_drain(drain_bar, status);   // every MMA issued has finished
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (EPI_WARPS warps)
        const int ew = warp - 2;
        const int quarter = warp & 3;             // TMEM lane quarter this warp may access
        const int half = ew >> 2;                 // which 128 of the 256 columns
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
            const Tile tl = decode(ts, gt, dir, t);
            const int l = gt.l[tl.g];
            const KRange kr = kranges(dir, tl.rt, n_extra(l), ts.KB);
            const int nkb = kr.count();
            const int nl = gt.line0[tl.g + 1] - gt.line0[tl.g];
            const int row = tl.rt * BM + quarter * 32 + lane;
            const int cbase = tl.ct * BN_MAX + half * 128;     // first line of this thread's columns
            const int ncols = min(128, nl - cbase);           // may be <= 0
            const int nch = (tl.nmma > half * 128) ? ((min(tl.nmma - half * 128, 128) + 31) >> 5) : 0;
            const uint32_t tl_addr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * 128);
            float acc[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) acc[j] = 0.f;
            bool ok = true;
            for (int c0 = 0; c0 < nkb; c0 += KC) {
                if (!warp_all(mbar_wait(main_full, mphase, abort_flag, status, spin))) { ok = false; break; }
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
            float2 ph = make_float2(1.f, 0.f);
            if (ep.phase) ph = ep.per_l ? ep.phase[(size_t)l * N + row] : ep.phase[(size_t)(l & 1) * N + phase_entry(l, row, N)];
            if (ep.mode == kOutUserC64) {
                float2* o = reinterpret_cast<float2*>(ep.out0);
                const size_t chan_base = (size_t)gt.chan0[tl.g] + (cbase >> 1);
#pragma unroll
                for (int j = 0; j < 128; j += 2)
                    if (j < ncols) o[(chan_base + (j >> 1)) * N + row] = make_float2(acc[j], acc[j + 1]);
            } else if (ep.mode == kOutUserF32) {
                const size_t chan_base = (size_t)gt.chan0[tl.g] + cbase;
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (j < ncols) ep.out0[(chan_base + j) * N + row] = acc[j];
            } else if (ep.mode == kOutPlanarF32) {
                const size_t line_base = (size_t)gt.line0[tl.g] + cbase;
#pragma unroll
                for (int j = 0; j < 128; ++j)
                    if (j < ncols) ep.out0[(line_base + j) * N + row] = acc[j];
            } else {   // kOutPlanarSplit: complex pairs with optional phase, TF32 split
                const size_t line_base = (size_t)gt.line0[tl.g] + cbase;
#pragma unroll
                for (int j = 0; j < 128; j += 2) {
                    if (j < ncols) {
                        const float re = acc[j] * ph.x - acc[j + 1] * ph.y;
                        const float im = acc[j] * ph.y + acc[j + 1] * ph.x;
                        const float hr = round_tf32(re), hi = round_tf32(im);
                        const size_t o = (line_base + j) * N + row;
                        ep.out0[o] = hr;
                        ep.out1[o] = round_tf32(re - hr);
                        ep.out0[o + N] = hi;
                        ep.out1[o + N] = round_tf32(im - hi);
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

}  // namespace

unsigned tc_default_spin_limit() { return tc::kSpinLimit; }

int contract_tf32x3(const dsbt_plan* p, const GroupTable& g, int dir, const float* in_hi,
                    const float* in_lo, int out_mode, float* out0, float* out1, const float2* phase,
                    int* sched, cudaStream_t st) {
    if (!p->has_tmaps) {
        set_error("split-TF32 path needs a plan built with DSBT_PLAN_TF32X3");
        return DSBT_ERR_UNSUPPORTED;
    }
    const int N = p->N;
    TileSpace ts;
    ts.RT = N / BM;
    ts.KB = N / BK;
    ts.t0[0] = 0;
    for (int i = 0; i < g.ngroups; ++i) {
        const int gi = g.ngroups - 1 - i;   // largest l first
        const int nl = g.line0[gi + 1] - g.line0[gi];
        ts.order[i] = gi;
        ts.ct[i] = (nl + BN_MAX - 1) / BN_MAX;
        ts.t0[i + 1] = ts.t0[i] + ts.RT * ts.ct[i];
    }
    ts.total = ts.t0[g.ngroups];
    if (ts.total == 0) return DSBT_OK;
    if (out_mode == kOutPlanarSplit || out_mode == kOutUserC64) {
        for (int i = 0; i < g.ngroups; ++i) {
            if ((g.line0[i] & 1) || ((g.line0[i + 1] - g.line0[i]) & 1)) {
                set_error("complex output needs whole channels per group");
                return DSBT_ERR_INVALID;
            }
        }
    }
    CUtensorMap tb_hi, tb_lo;
    int rc = encode_tmap_f32_sw128(&tb_hi, in_hi, (uint64_t)g.total_lines, N, BBOX, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f32_sw128(&tb_lo, in_lo, (uint64_t)g.total_lines, N, BBOX, BK);
    if (rc != DSBT_OK) return rc;
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 256;
    rc = ensure_smem((const void*)k_contract_tf32x3, smem);
    if (rc) return rc;
    int dev = 0, nsm = 0;
    DSBT_CUDA_TRY(cudaGetDevice(&dev));
    DSBT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = ts.total < nsm ? ts.total : nsm;
    EpiArgs ep{out_mode, out0, out1, phase, p->knl != nullptr};
    const CUtensorMap& ahi = dir > 0 ? p->tm_T_hi : p->tm_Tt_hi;
    const CUtensorMap& alo = dir > 0 ? p->tm_T_lo : p->tm_Tt_lo;
    DSBT_CUDA_TRY(cudaMemsetAsync(sched, 0, sizeof(int), st));
    ProfScope ps(kKContractTF32, st);
    k_contract_tf32x3<<<grid, NTHREADS, smem, st>>>(ahi, alo, tb_hi, tb_lo, g, ts, N, dir, ep, p->status,
                                                    p->spin_limit, sched);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

}  // namespace dsbt
