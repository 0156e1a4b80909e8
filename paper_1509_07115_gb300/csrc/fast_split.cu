// fast_split.cu -- split-precision tensor-core contractions with T_l and T_l^T
// in O(N l log N) work, for plans built with DSBT_PLAN_FAST_SPLIT (the stable
// counterpart of the fast scheme of Sec. 2.6, on tcgen05).
//
// Operands are FP16 pairs hi + lo (11 significant bits each, as TF32, at twice
// the TF32 tensor rate and half the bytes): plan factors scaled by 2^14 (rows of
// an orthogonal matrix, |entries| <= 1), lines scaled per channel by a power of
// two 2^e with ||2^e psi|| < 2^13 (set by the sine/cosine kernel or the input
// split), so every intermediate of the orthogonal maps stays far inside the
// FP16 range and the FP16 subnormal step lies 2^-36 below the channel norm.
// Each K step issues hi*hi + hi*lo + lo*hi into one FP32 TMEM accumulator
// (lo*lo, 2^-22 relative, dropped); epilogues remove 2^14 (and 2^e where the
// output leaves the scaled domain) by exact power-of-two products.
//
// On a regular row n of T_l the entries left of the diagonal are
// T_nm = alpha_n P'_l(n - m, 2n) sqrt(w_m): a polynomial of degree l - 1 in m
// times sqrt(w_m) (Sec. 2.4, Eqs. (38)-(42)).  Columns are cut into leaves of
// 128 (one output row tile) and a binary tree of intervals above them.  An
// interval (j, i) of 128 * 2^j columns is "used" when i is even and its right
// sibling i + 1 exists: the rows of that sibling take it as a far interval, and
// every row r of leaf J takes exactly the used intervals ((J >> j) - 1) for the
// set bits j of J.  On a used interval the row is sqrt(w) (Q_j beta_{r,j}) with
// Q_j an orthonormal basis [len][64] of the polynomials of degree < 64 on the
// interval's points.  Used intervals are numbered (slots s, level-major); the
// augmented index (s, k), k < 64, spans NA = 64 (nleaf - 1) columns.
//
// Every step is then the contraction of gemm_tf32x3.cu with other operands and
// K ranges.  Tiles are short (4-16 K blocks), so the TMEM accumulator is split
// into two 256-column buffers used by alternate chunks of KC K blocks (all three
// split products of a chunk into one buffer): the MMAs of the next chunk, also
// across tiles, run while the epilogue drains the previous one.
//   forward   MOMENTS  M[line][(s,k)]  = sum_t QT[(s,k)][t] f[line][t]          (t in interval s)
//             EVAL     b[line][r]      = sum_c T[r][c] f[line][c]  (near band: c in r's leaf)
//                                      + sum_(s,k) B[r][(s,k)] M[line][(s,k)]  (far slots of r)
//   inverse   WEIGHTS  W[line][(s,k)]  = sum_r BT[(s,k)][r] b[line][r]          (r in sibling of s)
//             LEAFOUT  f[line][c]      = sum_r T^T[c][r] b[line][r] (completion rows and near band)
//                                      + sum_(s,k) QA[c][(s,k)] W[line][(s,k)]  (used slots holding c)
// The completion rows n < n0_l (Sec. 2.5) are polynomials of degree < l in m
// too, so the forward gives them the columns right of leaf 0 through extra
// "right" slots: the intervals (j, 1), j = 0 .. levels - 1.
// With B[r][(s,k)] = beta_{r,j}[k] (zero unless s is a far slot of r), BT its
// transpose, QT[(s,k)][t] = Q_j[t - i len][k] sqrt(w_t) and QA its transpose,
// all split into FP16 pairs.  MOMENTS and WEIGHTS tiles hold two slots (64
// rows of QT / BT each; a slot of odd level with the child slot whose range it
// contains, else two slots of similar length).  K blocks of a tile come from up to two operand
// sources (near: T / T^T against the lines; far: B / QA against M / W), listed
// per tile by segments.  Each direction is one persistent launch over both
// kinds of tiles: a row tile loads its near band first, then waits (bounded,
// on a per-unit device counter that the moment tiles' epilogue warps raise
// after their stores) before it loads the augmented lines.
//
// Work per line (N = 4096, l = 63): near 0.5 M, far 0.7 M, moments 1.3 M (half
// of it on the ignored lanes), leaf 0 0.5 M multiply-adds, against 8.7 M for the
// dense tiles: about 3x fewer tensor operations.
#include <math.h>

#include <algorithm>
#include <thread>
#include <vector>

#include <cuda_fp16.h>

#include "plan.cuh"
#include "tc_ptx.cuh"

namespace dsbt {

namespace {

using namespace tc;

constexpr int BM = 128;
constexpr int BK = 64;                             // K elements per block: one 128-byte swizzle row of FP16
constexpr int BN_MAX = 256;
constexpr int BBOX = 256;                          // rows per B TMA box (one box per operand half; 64 and 128: 1 % slower)
constexpr int STAGES = 2;
// K blocks per chunk.  The tensor cores accumulate with truncation, and all
// three split products of a chunk go into one buffer, so the chunk is one K
// block: the round-trip error at N = 4096, l <= 63 is then 5.6e-7, the dense
// kernel's (2 blocks: 8.3e-7; a separate correction accumulator, as in the
// dense kernel, leaves no TMEM columns for a second buffer).
constexpr int KC = 1;
constexpr int EPI_WARPS = 8;                       // two per TMEM lane quarter
constexpr int WC = BN_MAX * 4 / EPI_WARPS;         // accumulator columns per epilogue warp
constexpr int QS = 4;                              // tile-queue slots
constexpr int A_BYTES = BM * BK * 2;               // 16 KiB
constexpr int B_BYTES = BN_MAX * BK * 2;           // 32 KiB
constexpr float kFacScale = 16384.f;               // plan factors are stored times 2^14
constexpr float kFacUnscale = 1.f / 16384.f;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int NTHREADS = 64 + 32 * EPI_WARPS;
constexpr int FL = 128;                            // leaf = output row tile
constexpr int KP = 64;                             // basis functions per interval (>= l_max)
constexpr int MAX_LEVELS = 6;                      // N / 128 <= 64 (plans have N <= 8192)
constexpr int MAX_SLOTS = (1 << MAX_LEVELS) - 1;
constexpr int MAX_RIGHT = 2 * MAX_LEVELS;          // intervals covering the columns right of leaf 0
constexpr int MAX_FSLOTS = MAX_SLOTS + MAX_RIGHT;
constexpr int MAX_SEGS = MAX_RIGHT + 2;
// Default: the plain order (every first-kind tile, then every second-kind
// tile).  A short lag makes row tiles wait: the longest moment tiles stream
// about 3 MB of lines each, tens of microseconds at one SM's share of the HBM
// rate, while the whole GPU finishes a unit in about 4 us, so a row tile
// trails its unit by 16 or more units to find it done, and that many units'
// lines no longer fit in L2 (N = 4096, l <= 63 x 8: lag 16 is 12 % slower
// than the plain order, lag 4 2x).
constexpr int kDefaultLag = 1 << 30;

enum Mode { kMoments = 0, kEval = 1, kWeights = 2, kLeafOut = 3 };

struct FtcSpace {
    int amode;                     // first kind of this launch: kMoments (forward) or kWeights (adjoint)
    int omode;                     // second kind: kEval (forward) or kLeafOut (adjoint)
    int kc;                        // K blocks per main-accumulator chunk
    int RT;                        // row tiles of a second-kind unit (the leaves)
    int KB;                        // K blocks of N
    int nleaf, levels, nslots;     // leaves of 128 (any count 2..64), tree levels, used slots
    int nslots_f;                  // forward slots: the used ones, then the right intervals
    int nright;                    // right intervals (rj, ri): the columns right of leaf 0
    int rj[MAX_RIGHT], ri[MAX_RIGHT];
    int FW;                        // slots per row of the compact B table: max(levels, nright)
    int a_oob;                     // a row past the end of the MOMENTS / WEIGHTS A operand
    int slot_off[MAX_LEVELS + 1];  // first slot of level j
    int npairs;                    // MOMENTS / WEIGHTS tiles of a unit: slot pairs (b = -1: single slot)
    int pair_a[MAX_FSLOTS], pair_b[MAX_FSLOTS];
    // A unit is one column tile (BN_MAX lines) of one group.  Units are numbered
    // group by group (largest l first); unit u's first-kind tiles come before
    // its second-kind tiles, which read what they wrote, and the launch runs
    // block k = [first kind of unit k] [second kind of unit k - lag], so the
    // second pass over a unit's lines finds them (and its fresh augmented
    // lines) in L2.
    int npos;                      // groups of the launch
    int units;                     // U
    int lag;                       // 1 <= lag <= U
    int total;                     // tiles
    int order[kMaxGroups];         // group at position i
    int u0[kMaxGroups + 1];        // first unit of position i
    int acum[kMaxGroups + 1];      // first-kind tiles before position i
    int ta[kMaxGroups];            // first-kind tiles per unit at position i (npairs, or 0 for l = 0)
};

struct Tile {
    int g, rt, ct, nmma, mode, unit, wait;   // mode < 0: no more tiles
};

// Position of unit u (u0 is increasing).
__device__ __forceinline__ int unit_pos(const FtcSpace& fs, int u) {
    int lo = 0, hi = fs.npos;   // u0[lo] <= u < u0[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (fs.u0[mid] <= u) lo = mid;
        else hi = mid;
    }
    return lo;
}

// First tile of block k < U, a block of position i.
__device__ __forceinline__ int block_start(const FtcSpace& fs, int i, int k) {
    return fs.acum[i] + (k - fs.u0[i]) * fs.ta[i] + fs.RT * max(0, k - fs.lag);
}

// Tile t -> (kind, unit, row tile or pair, group, column tile): the last block
// k whose first tile is <= t (blocks may be empty), found by a search over the
// positions, then over the position's units; blocks k >= U hold second-kind
// tiles only.
__device__ __forceinline__ Tile decode(const FtcSpace& fs, const GroupTable& gt, int t) {
    const int tail = fs.acum[fs.npos];   // first-kind tiles of the launch
    int k, na = 0;
    if (t >= tail + fs.RT * max(0, fs.units - fs.lag)) {
        k = fs.lag + (t - tail) / fs.RT;
    } else {
        int lo = 0, hi = fs.npos;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (block_start(fs, mid, fs.u0[mid]) <= t) lo = mid;
            else hi = mid;
        }
        const int i = lo;
        int a = fs.u0[i], c = fs.u0[i + 1];   // block_start(a) <= t < block_start(c)
        while (c - a > 1) {
            const int mid = (a + c) >> 1;
            if (block_start(fs, i, mid) <= t) a = mid;
            else c = mid;
        }
        k = a;
        na = fs.ta[i];
    }
    const int start = k < fs.units ? block_start(fs, unit_pos(fs, k), k) : tail + fs.RT * (k - fs.lag);
    int local = t - start;
    Tile tl;
    if (local < na) {
        tl.mode = fs.amode;
        tl.unit = k;
        tl.rt = local;   // pairs are sorted longest first
    } else {
        local -= na;
        tl.mode = fs.omode;
        tl.unit = k - fs.lag;
        if (fs.omode == kEval) tl.rt = (local == 0) ? 0 : fs.RT - local;   // dense leaf 0 first
        else tl.rt = local;
    }
    const int i = unit_pos(fs, tl.unit);
    const int g = fs.order[i];
    tl.g = g;
    tl.ct = tl.unit - fs.u0[i];
    tl.wait = tl.mode == fs.omode && fs.ta[i] > 0;   // the unit has first-kind tiles
    const int nl = gt.line0[g + 1] - gt.line0[g];
    int left = nl - tl.ct * BN_MAX;
    if (left > BN_MAX) left = BN_MAX;
    tl.nmma = (left + 15) & ~15;
    return tl;
}

// Intervals of level j that start inside the grid (the last may end past it).
__host__ __device__ inline int n_at(const FtcSpace& fs, int j) { return (fs.nleaf + (1 << j) - 1) >> j; }

// Interval (j, i) is "used" (has a slot) when i is even and its right sibling
// starts inside the grid: the rows of that sibling take it as a far interval.
__host__ __device__ inline bool used(const FtcSpace& fs, int j, int i) { return (i & 1) == 0 && i + 1 < n_at(fs, j); }

// slot s -> (level j, interval i); slots s >= nslots (forward only) are the
// right intervals (rj, ri) that cover the columns right of leaf 0 for the
// completion rows.
__host__ __device__ inline void slot_ji(const FtcSpace& fs, int s, int& j, int& i) {
    if (s >= fs.nslots) {
        j = fs.rj[s - fs.nslots];
        i = fs.ri[s - fs.nslots];
        return;
    }
    j = 0;
    while (j + 1 < fs.levels && fs.slot_off[j + 1] <= s) ++j;
    i = 2 * (s - fs.slot_off[j]);
}

// K blocks [k0, k1) a MOMENTS (the interval's columns) or WEIGHTS (its
// sibling's rows) slot contracts over.
__device__ __forceinline__ void aug_range(const FtcSpace& fs, int mode, int s, int& k0, int& k1) {
    int j, i;
    slot_ji(fs, s, j, i);
    const int lb = (FL << j) / BK;
    k0 = (mode == kMoments) ? i * lb : (i + 1) * lb;
    k1 = min(k0 + lb, fs.KB);   // a sibling at the right edge may end past the grid
}

// K blocks of one tile: segments [k0, k1) of operand source src (1 near: the
// lines against a diagonal 128 x 128 block of T_l / T_l^T or, for MOMENTS and
// WEIGHTS, the basis rows; 2 far: the augmented lines against B / QA; 3: the
// completion block, T_l rows < 64 transposed, against the lines' K block 0).
// The B operand's K block is kb; the A operand's is ak + (kb - k0) (A tables
// that are stored compactly index K differently from the lines).
struct Segs {
    int n;
    int src[MAX_SEGS], k0[MAX_SEGS], k1[MAX_SEGS], ak[MAX_SEGS];
    __device__ __forceinline__ void add(int s, int a, int b, int a_k) {
        if (b > a) {
            src[n] = s;
            k0[n] = a;
            k1[n] = b;
            ak[n] = a_k;
            ++n;
        }
    }
    __device__ __forceinline__ int count() const {
        int c = 0;
        for (int q = 0; q < n; ++q) c += k1[q] - k0[q];
        return c;
    }
    __device__ __forceinline__ void at(int i, int& s, int& kb, int& akb) const {
        for (int q = 0; q < n; ++q) {
            const int len = k1[q] - k0[q];
            if (i < len) {
                s = src[q];
                kb = k0[q] + i;
                akb = ak[q] + i;
                return;
            }
            i -= len;
        }
        s = 1;
        kb = 0;
        akb = 0;
    }
};

__device__ __forceinline__ Segs segments(const FtcSpace& fs, int mode, int l, int rt) {
    Segs sg;
    sg.n = 0;
    const int nx = n_extra(l);
    const int nf = (l + BK - 1) / BK;   // far K blocks per slot (basis functions k < l)
    constexpr int SB = KP / BK;         // K blocks per slot
    if (mode == kMoments || mode == kWeights) {
        // the K ranges of the tile's two slots are dyadic intervals: nested
        // (one segment, the larger) or disjoint (two segments)
        int a0, a1, b0 = 0, b1 = 0;
        aug_range(fs, mode, fs.pair_a[rt], a0, a1);
        if (fs.pair_b[rt] >= 0) aug_range(fs, mode, fs.pair_b[rt], b0, b1);
        if (b1 <= b0 || (b0 >= a0 && b1 <= a1)) {
            sg.add(1, a0, a1, a0);
        } else if (a0 >= b0 && a1 <= b1) {
            sg.add(1, b0, b1, b0);
        } else {
            sg.add(1, a0, a1, a0);
            sg.add(1, b0, b1, b0);
        }
    } else if (mode == kEval) {
        // A: the leaf's diagonal block (K blocks 0, 1) and the compact B table,
        // whose slot q of a row is the far interval at level q (regular rows)
        // or right interval q (completion rows).  The near band comes first:
        // its loads need nothing from this launch's first kind.
        if (rt == 0) {
            // leaf 0: near band; the completion rows (polynomials of degree < l
            // in m as well) take the columns right of it through the right slots
            sg.add(1, 0, FL / BK, 0);
            if (nx > 0)
                for (int q = 0; q < fs.nright; ++q) {
                    const int s = fs.nslots + q;
                    sg.add(2, s * SB, s * SB + nf, q * SB);
                }
        } else {
            sg.add(1, rt * (FL / BK), (rt + 1) * (FL / BK), 0);
            for (int j = 0; j < fs.levels; ++j)
                if ((rt >> j) & 1) {
                    const int s = fs.slot_off[j] + (((rt >> j) - 1) >> 1);
                    sg.add(2, s * SB, s * SB + nf, j * SB);
                }
        }
    } else {   // kLeafOut: A = the transposed diagonal block, the completion block, QA (dense)
        if (rt > 0 && nx > 0) sg.add(3, 0, 1, 0);   // completion rows n < n0_l (storage rows < 64)
        sg.add(1, rt * (FL / BK), (rt + 1) * (FL / BK), 0);
        for (int j = 0; j < fs.levels; ++j) {
            const int i = rt >> j;
            if (used(fs, j, i)) {
                const int s = fs.slot_off[j] + (i >> 1);
                sg.add(2, s * SB, s * SB + nf, s * SB);
            }
        }
    }
    return sg;
}

// Number of K blocks of a tile (what segments(...).count() gives), without
// building the list.
__device__ __forceinline__ int seg_count(const FtcSpace& fs, int mode, int l, int rt) {
    const int nx = n_extra(l);
    const int nf = (l + BK - 1) / BK;
    if (mode == kMoments || mode == kWeights) {
        int a0, a1, b0 = 0, b1 = 0;
        aug_range(fs, mode, fs.pair_a[rt], a0, a1);
        if (fs.pair_b[rt] >= 0) aug_range(fs, mode, fs.pair_b[rt], b0, b1);
        if (b1 <= b0 || (b0 >= a0 && b1 <= a1)) return a1 - a0;
        if (a0 >= b0 && a1 <= b1) return b1 - b0;
        return (a1 - a0) + (b1 - b0);
    }
    if (mode == kEval) return rt == 0 ? FL / BK + (nx > 0 ? fs.nright * nf : 0) : __popc(rt) * nf + FL / BK;
    int c = ((rt > 0 && nx > 0) ? 1 : 0) + FL / BK;
    for (int j = 0; j < fs.levels; ++j)
        if (used(fs, j, rt >> j)) c += nf;
    return c;
}

struct EpiArgs {
    int mode;              // OutMode of the second kind's output
    void* out0;            // FP16 pair (kOutPlanarSplit) or FP32 values
    void* out1;
    const float2* phase;
    int per_l;
    const float* scale;    // per line: 2^-e, the factor that leaves the scaled domain
    __half* aug0;          // the first kind's output, the augmented lines [line][astride] (FP16 pair)
    __half* aug1;
    int astride;
};

// FP16 pair of v: hi = fp16(v), lo = fp16(v - hi).
__device__ __forceinline__ void split_f16(float v, __half& hi, __half& lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}
// Barriers, the tile queue and two words after the stages (the launch adds
// 512 bytes past the 1024-byte alignment of the stages).
static_assert((2 * STAGES + 4 + 2 * QS + 1) * 8 + QS * sizeof(Tile) + 8 <= 512, "control area");

// Counter block of a launch (zeroed before it): the tile scheduler, the
// launch-wide abort word and, per unit, the first-kind epilogue warps done.
constexpr int kCtrSched = 0, kCtrAbort = 1, kCtrUnits = 2;

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Orders this thread's generic-proxy global accesses with its async-proxy
// (TMA) ones.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// A second-kind tile's producer waits, before its first load of augmented
// lines, until every first-kind epilogue warp of its unit has stored its part:
// at most `spin` polls, and it gives up at once when this CTA or another one
// aborted.  The first-kind tiles of a unit come earlier in the tile order and
// need nothing from later tiles, so the wait ends while the hardware runs.
__device__ __forceinline__ bool wait_unit(const int* cnt, int target, const int* gabort, volatile int* abort_flag,
                                          unsigned* status, uint32_t spin) {
    for (uint32_t it = 0; it < spin; ++it) {
        if (ld_acquire(cnt) >= target) {
            fence_proxy_async_global();   // the TMA loads that follow see the stores
            return true;
        }
        if (*abort_flag || *(volatile const int*)gabort) {
            *abort_flag = 1;
            return false;
        }
        __nanosleep(64);
    }
    *abort_flag = 1;
    atomicExch(status, (unsigned)kStatusTimeout);
    return false;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// The kernel: roles and bounded waits as in gemm_tf32x3.cu; what differs is
// where each K block comes from, the two kinds of tiles in one launch and the
// two alternating accumulator buffers.
__global__ void __launch_bounds__(NTHREADS, 1)
k_contract_ftc(const __grid_constant__ CUtensorMap tmA0_hi, const __grid_constant__ CUtensorMap tmA0_lo,
               const __grid_constant__ CUtensorMap tmA1_hi, const __grid_constant__ CUtensorMap tmA1_lo,
               const __grid_constant__ CUtensorMap tmB1_hi, const __grid_constant__ CUtensorMap tmB1_lo,
               const __grid_constant__ CUtensorMap tmA2_hi, const __grid_constant__ CUtensorMap tmA2_lo,
               const __grid_constant__ CUtensorMap tmB2_hi, const __grid_constant__ CUtensorMap tmB2_lo,
               const __grid_constant__ CUtensorMap tmA3_hi, const __grid_constant__ CUtensorMap tmA3_lo,
               GroupTable gt, FtcSpace fs, int N, EpiArgs ep, unsigned* status, uint32_t spin, int* ctr) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* stage_base = smem;
    uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
    uint64_t* empty = full + STAGES;
    uint64_t* acc_full = empty + STAGES;    // [2]: a chunk's sum is in TMEM buffer b
    uint64_t* acc_empty = acc_full + 2;     // [2]: buffer b drained by the epilogue
    uint64_t* tq_full = acc_empty + 2;
    uint64_t* tq_empty = tq_full + QS;
    uint64_t* drain_bar = tq_empty + QS;    // the MMA issuer's exit drain
    Tile* tile_q = (Tile*)(drain_bar + 1);   // decoded by the producer for the other roles
    uint32_t* tmem_slot = (uint32_t*)(tile_q + QS);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int unit_target = fs.npairs * EPI_WARPS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], EPI_WARPS);
        }
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
            // the first kind's lines are read again by the second kind, and the
            // augmented lines by several row tiles: keep them; a row tile's
            // near band is the last use of its lines
            const uint64_t pol_keep = policy_evict_last(), pol_last = policy_evict_first();
            int qslot = 0;
            uint32_t qphase = 0;
            while (ok) {
                if (!mbar_wait(&tq_empty[qslot], qphase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                const int t = atomicAdd(ctr + kCtrSched, 1);
                Tile tl;
                if (t < fs.total) tl = decode(fs, gt, t);
                else tl.mode = -1;
                tile_q[qslot] = tl;
                mbar_arrive(&tq_full[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (tl.mode < 0) break;
                const bool aug = tl.mode == fs.amode;   // two slots per tile, 64 A rows each
                const int l = gt.l[tl.g];
                const Segs sg = segments(fs, tl.mode, l, tl.rt);
                const int nbox = (tl.nmma + BBOX - 1) / BBOX;
                const bool pair = aug && fs.pair_b[tl.rt] >= 0;
                const uint32_t a_bytes = (aug ? 64u : 128u) * BK * 2u;
                const uint32_t bytes = 2 * a_bytes * (pair ? 2 : 1) + 2 * nbox * BBOX * BK * 2;
                int arow1, arow2 = 0;
                int ra0 = 0, ra1 = 0, rb0 = 0, rb1 = 0;   // own K ranges of the two slots
                if (aug) {
                    aug_range(fs, tl.mode, fs.pair_a[tl.rt], ra0, ra1);
                    if (pair) aug_range(fs, tl.mode, fs.pair_b[tl.rt], rb0, rb1);
                }
                if (tl.mode == kMoments) {
                    arow1 = ((l & 1) * fs.nslots_f + fs.pair_a[tl.rt]) * KP;
                    if (pair) arow2 = ((l & 1) * fs.nslots_f + fs.pair_b[tl.rt]) * KP;
                } else if (tl.mode == kWeights) {   // compact BT: rows (l, level, k)
                    int j, i;
                    slot_ji(fs, fs.pair_a[tl.rt], j, i);
                    arow1 = (l * fs.levels + j) * KP;
                    if (pair) {
                        slot_ji(fs, fs.pair_b[tl.rt], j, i);
                        arow2 = (l * fs.levels + j) * KP;
                    }
                } else {
                    arow1 = (l * fs.nleaf + tl.rt) * BM;   // diagonal block of leaf rt
                    arow2 = (tl.mode == kEval ? l : (l & 1)) * N + tl.rt * BM;
                }
                const int brow = gt.line0[tl.g] + tl.ct * BN_MAX;
                const int nkb = sg.count();
                bool waited = !tl.wait;
                for (int i = 0; i < nkb; ++i) {
                    int src, kb, akb;
                    sg.at(i, src, kb, akb);
                    if (src == 2 && !waited) {
                        if (!wait_unit(ctr + kCtrUnits + tl.unit, unit_target, ctr + kCtrAbort, abort_flag, status,
                                       spin)) { ok = false; break; }
                        waited = true;
                    }
                    if (!mbar_wait(&empty[stage], phase ^ 1, abort_flag, status, spin)) { ok = false; break; }
                    unsigned char* sb = stage_base + stage * STAGE_BYTES;
                    mbar_expect_tx(&full[stage], bytes);
                    led.arm(stage, phase);
                    const CUtensorMap* ah = aug ? &tmA0_hi : (src == 1 ? &tmA1_hi : (src == 2 ? &tmA2_hi : &tmA3_hi));
                    const CUtensorMap* al = aug ? &tmA0_lo : (src == 1 ? &tmA1_lo : (src == 2 ? &tmA2_lo : &tmA3_lo));
                    const CUtensorMap* bh = src == 2 ? &tmB2_hi : &tmB1_hi;
                    const CUtensorMap* bl = src == 2 ? &tmB2_lo : &tmB1_lo;
                    if (aug) {   // slot a -> A rows 0..63, slot b -> rows 64..127
                        // a slot's rows are loaded only on its own K range: elsewhere
                        // (the other slot of a disjoint pair) the load starts past the
                        // table's last row and the copy fills zeros
                        const int ya = (kb >= ra0 && kb < ra1) ? arow1 : fs.a_oob;
                        tma_load_2d(sb, ah, &full[stage], kb * BK, ya);
                        tma_load_2d(sb + A_BYTES, al, &full[stage], kb * BK, ya);
                        if (pair) {
                            const int yb = (kb >= rb0 && kb < rb1) ? arow2 : fs.a_oob;
                            tma_load_2d(sb + KP * 128, ah, &full[stage], kb * BK, yb);
                            tma_load_2d(sb + A_BYTES + KP * 128, al, &full[stage], kb * BK, yb);
                        }
                    } else {
                        // near: K block akb of the leaf's diagonal block; far: slot
                        // akb of the compact B table (forward) or augmented column
                        // kb of QA (adjoint); completion: T_l rows 0..63 of the leaf's
                        // columns
                        const int arow = src == 1 ? arow1 : (src == 2 ? arow2 : l * N + tl.rt * BM);
                        tma_load_2d(sb, ah, &full[stage], akb * BK, arow);
                        tma_load_2d(sb + A_BYTES, al, &full[stage], akb * BK, arow);
                    }
                    const uint64_t pol = (!aug && src == 1) ? pol_last : pol_keep;
                    for (int b = 0; b < nbox; ++b) {
                        tma_load_2d_hint(sb + 2 * A_BYTES + b * BBOX * 128, bh, &full[stage], kb * BK,
                                         brow + b * BBOX, pol);
                        tma_load_2d_hint(sb + 2 * A_BYTES + B_BYTES + b * BBOX * 128, bl, &full[stage],
                                         kb * BK, brow + b * BBOX, pol);
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
            uint32_t gch = 0;   // chunks issued so far: buffer gch & 1, round gch >> 1
            bool ok = true;
            int qslot = 0;
            uint32_t qphase = 0;
            while (ok) {
                if (!mbar_wait(&tq_full[qslot], qphase, abort_flag, status, spin)) break;
                const Tile tl = tile_q[qslot];
                mbar_arrive(&tq_empty[qslot]);
                if (++qslot == QS) { qslot = 0; qphase ^= 1; }
                if (tl.mode < 0) break;
                const int l = gt.l[tl.g];
                const int nkb = seg_count(fs, tl.mode, l, tl.rt);
                const uint32_t idesc = idesc_f16(BM, tl.nmma);
                for (int c0 = 0; c0 < nkb && ok; c0 += fs.kc) {
                    const int c1 = min(nkb, c0 + fs.kc);
                    const int buf = gch & 1;
                    // the epilogue drained this buffer's previous chunk; the other
                    // buffer may still be draining while these MMAs run
                    if (!mbar_wait(&acc_empty[buf], ((gch >> 1) & 1) ^ 1, abort_flag, status, spin)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)buf * 256;
                    uint32_t accf = 0;
                    for (int i = c0; i < c1; ++i) {
                        if (!mbar_wait(&full[stage], phase, abort_flag, status, spin)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t sa = smem_u32(stage_base + stage * STAGE_BYTES);
                        const uint32_t sa_lo = sa + A_BYTES;
                        const uint32_t sb_hi = sa + 2 * A_BYTES;
                        const uint32_t sb_lo = sb_hi + B_BYTES;
#pragma unroll
                        for (int ks = 0; ks < BK / 16; ++ks) {
                            const uint32_t off = ks * 32;   // 16 FP16 values = 32 bytes along K
                            const uint64_t dah = sdesc_sw128(sa + off), dal = sdesc_sw128(sa_lo + off);
                            const uint64_t dbh = sdesc_sw128(sb_hi + off), dbl = sdesc_sw128(sb_lo + off);
                            mma_f16(d, dah, dbh, idesc, accf);
                            mma_f16(d, dah, dbl, idesc, 1);
                            mma_f16(d, dal, dbh, idesc, 1);
                            accf = 1;
                        }
                        mma_commit(&empty[stage]);
                        if (++stage == STAGES) { stage = 0; phase ^= 1; }
                    }
                    if (!ok) break;
                    mma_commit(&acc_full[buf]);
                    ++gch;
                }
            }
            mma_drain(drain_bar, status);   // every MMA issued has finished
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue (EPI_WARPS warps)
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;   // column group of the warp: columns [half WC, (half + 1) WC)
        uint32_t gch = 0;   // chunks drained so far (same order as the MMA issuer)
        int qslot = 0;
        uint32_t qphase = 0;
        while (true) {
            if (!warp_all(mbar_wait(&tq_full[qslot], qphase, abort_flag, status, spin))) break;
            const Tile tl = tile_q[qslot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tq_empty[qslot]);
            if (++qslot == QS) { qslot = 0; qphase ^= 1; }
            if (tl.mode < 0) break;
            const bool aug = tl.mode == fs.amode;
            const int l = gt.l[tl.g];
            const int nkb = seg_count(fs, tl.mode, l, tl.rt);
            const int nl = gt.line0[tl.g + 1] - gt.line0[tl.g];
            const int trow = quarter * 32 + lane;                 // TMEM lane = A row of the tile
            int row = tl.rt * BM + trow;
            bool store_row = true;
            if (aug) {   // lanes 0..63: slot a, 64..127: slot b
                const int slot = trow < KP ? fs.pair_a[tl.rt] : fs.pair_b[tl.rt];
                store_row = slot >= 0;
                row = slot * KP + (trow & (KP - 1));
            }
            const int cbase = tl.ct * BN_MAX + half * WC;
            const int ncols = min(WC, nl - cbase);
            const int nch = (tl.nmma > half * WC) ? ((min(tl.nmma - half * WC, WC) + 31) >> 5) : 0;
            const uint32_t tl_addr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(half * WC);
            float acc[WC];
#pragma unroll
            for (int j = 0; j < WC; ++j) acc[j] = 0.f;
            bool ok = true;
            for (int c0 = 0; c0 < nkb; c0 += fs.kc) {
                const int buf = gch & 1;
                if (!warp_all(mbar_wait(&acc_full[buf], (gch >> 1) & 1, abort_flag, status, spin))) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int ch = 0; ch < WC / 32; ++ch) {
                    if (ch < nch) {
                        float v[32];
                        tmem_ld32(tl_addr + (uint32_t)buf * 256 + ch * 32, v);
#pragma unroll
                        for (int j = 0; j < 32; ++j) acc[ch * 32 + j] += v[j];
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
                ++gch;
            }
            if (!ok) break;
            const bool do_store = ncols > 0 && store_row;   // warp-uniform
            if (aug) {   // moments / weights stay in the scaled domain
                if (do_store) {
                    const int S = ep.astride;
                    __half* o0 = ep.aug0;
                    __half* o1 = ep.aug1;
                    const size_t line_base = (size_t)gt.line0[tl.g] + cbase;
#pragma unroll
                    for (int j = 0; j < WC; ++j) {
                        if (j < ncols) {
                            __half h, lo;
                            split_f16(acc[j] * kFacUnscale, h, lo);
                            const size_t o = (line_base + j) * S + row;
                            o0[o] = h;
                            o1[o] = lo;
                        }
                    }
                }
                // release this warp's part of the unit to the second kind's TMA loads
                fence_proxy_async_global();
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    atomicAdd(ctr + kCtrUnits + tl.unit, 1);
                }
                continue;
            }
            if (!do_store) continue;
            float2 ph = make_float2(1.f, 0.f);
            if (ep.phase) ph = ep.per_l ? ep.phase[(size_t)l * N + row] : ep.phase[(size_t)(l & 1) * N + phase_entry(l, row, N)];
            const size_t line_base = (size_t)gt.line0[tl.g] + cbase;
            if (ep.mode == kOutPlanarF32) {
                float* o = reinterpret_cast<float*>(ep.out0);
#pragma unroll
                for (int j = 0; j < WC; ++j)
                    if (j < ncols) o[(line_base + j) * N + row] = acc[j] * (ep.scale[line_base + j] * kFacUnscale);
            } else if (ep.mode == kOutUserC64) {
                float2* o = reinterpret_cast<float2*>(ep.out0);
                const size_t chan_base = (size_t)gt.chan0[tl.g] + (cbase >> 1);
                if (gt.uoff) {   // channels gathered by offset (uneven batch)
#pragma unroll
                    for (int j = 0; j < WC; j += 2)
                        if (j < ncols) {
                            const float u = ep.scale[line_base + j] * kFacUnscale;
                            o[(size_t)gt.uoff[chan_base + (j >> 1)] + row] = make_float2(acc[j] * u, acc[j + 1] * u);
                        }
                } else {
#pragma unroll
                    for (int j = 0; j < WC; j += 2)
                        if (j < ncols) {
                            const float u = ep.scale[line_base + j] * kFacUnscale;
                            o[(chan_base + (j >> 1)) * N + row] = make_float2(acc[j] * u, acc[j + 1] * u);
                        }
                }
            } else if (ep.mode == kOutUserF32) {
                float* o = reinterpret_cast<float*>(ep.out0);
                const size_t chan_base = (size_t)gt.chan0[tl.g] + cbase;
#pragma unroll
                for (int j = 0; j < WC; ++j)
                    if (j < ncols) {
                        const size_t at = gt.uoff ? (size_t)gt.uoff[chan_base + j] : (chan_base + j) * N;
                        o[at + row] = acc[j] * (ep.scale[line_base + j] * kFacUnscale);
                    }
            } else {   // kOutPlanarSplit: complex pairs with optional phase, FP16 pair, still scaled
                __half* o0 = reinterpret_cast<__half*>(ep.out0);
                __half* o1 = reinterpret_cast<__half*>(ep.out1);
#pragma unroll
                for (int j = 0; j < WC; j += 2) {
                    if (j < ncols) {
                        const float re = (acc[j] * ph.x - acc[j + 1] * ph.y) * kFacUnscale;
                        const float im = (acc[j] * ph.y + acc[j + 1] * ph.x) * kFacUnscale;
                        const size_t o = (line_base + j) * N + row;
                        __half h, lo;
                        split_f16(re, h, lo);
                        o0[o] = h;
                        o1[o] = lo;
                        split_f16(im, h, lo);
                        o0[o + N] = h;
                        o1[o + N] = lo;
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (threadIdx.x == 0 && *abort_flag) atomicExch(ctr + kCtrAbort, 1);   // waiters elsewhere give up
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
}

// ------------------------------------------------------------ plan data

// FP16 pair of a plan entry v stored times 2^14: hi = fp16(2^14 v),
// lo = fp16(2^14 v - hi), both rounded to nearest.
__device__ __forceinline__ void fac_pair(double v, __half& hi, __half& lo) {
    const double x = v * (double)kFacScale;
    hi = __double2half(x);
    lo = __double2half(x - (double)__half2float(hi));
}

// beta_{r,j}[k] of every row r of the used slot s = (j, i) it takes (the rows
// of the sibling interval i + 1 inside the grid), from the FP64 T_l:
//   beta = sum_t Q_j[t][k] T_l[r][i len + t] / sqrt(w_{i len + t}),
// zero on completion rows and for k >= l; written as FP16 pairs to the compact
// tables B[l][r][j][k] (a row takes at most one far interval per level) and
// BT[l][j][k][r].  Block (position, l), KP threads (k).
__global__ void k_ftc_beta(const double* __restrict__ T64, const double* __restrict__ Q,
                           const size_t* __restrict__ qoff, FtcSpace fs, int N, __half* bA_hi, __half* bA_lo,
                           __half* bT_hi, __half* bT_lo) {
    // positions q < N per level: the used slots of a level span fewer than N
    // columns (N / 2 when N / 128 is a power of two)
    const int j = blockIdx.x / N, q = blockIdx.x % N, l = blockIdx.y, k = threadIdx.x;
    const int len = FL << j;
    const int i = 2 * (q / len);
    const int r = (i + 1) * len + q % len;
    if (!used(fs, j, i) || r >= N) return;
    double b = 0.0;
    if (r >= n_extra(l) && k < l) {
        const double* row = T64 + ((size_t)l * N + r) * N + (size_t)i * len;
        const double* Qj = Q + qoff[j];
        for (int t = 0; t < len; ++t) {
            const double w = ((l & 1) && i == 0 && t == 0) ? 0.70710678118654752440 : 1.0;
            b = fma(row[t] / w, Qj[(size_t)t * KP + k], b);
        }
    }
    __half h, lo;
    fac_pair(b, h, lo);
    const size_t oa = (((size_t)l * N + r) * fs.FW + j) * KP + k;
    const size_t ot = (((size_t)l * fs.levels + j) * KP + k) * N + r;
    bA_hi[oa] = h;
    bA_lo[oa] = lo;
    bT_hi[ot] = h;
    bT_lo[ot] = lo;
}

// QT[p][(s,k)][c] = QA[p][c][(s,k)] = Q_j[c - i len][k] sqrt(w_c) for the
// columns c of used slot s = (j, i); parity p = 1 (odd l) carries
// sqrt(w_0) = 1/sqrt(2).  Block (position, p), KP threads (k).
__global__ void k_ftc_q(const double* __restrict__ Q, const size_t* __restrict__ qoff, FtcSpace fs, int N,
                        __half* qT_hi, __half* qT_lo, __half* qA_hi, __half* qA_lo) {
    const int j = blockIdx.x / N, q = blockIdx.x % N, p = blockIdx.y, k = threadIdx.x;
    const int len = FL << j;
    const int i = 2 * (q / len), t = q % len;
    if (!used(fs, j, i)) return;
    const int s = fs.slot_off[j] + q / len;
    const int c = i * len + t;
    const int NA = fs.nslots * KP;
    const double v = Q[qoff[j] + (size_t)t * KP + k] * ((p == 1 && c == 0) ? 0.70710678118654752440 : 1.0);
    __half h, lo;
    fac_pair(v, h, lo);
    const size_t ot = (((size_t)p * fs.nslots_f + s) * KP + k) * N + c;
    const size_t oa = ((size_t)p * N + c) * NA + (size_t)s * KP + k;
    qT_hi[ot] = h;
    qT_lo[ot] = lo;
    qA_hi[oa] = h;
    qA_lo[oa] = lo;
}

// Right intervals q = (rj, ri): beta of the completion rows r < n0_l - p_l on
// the columns [ri len, (ri + 1) len) (all right of leaf 0, weight 1) into
// B[l][r][q][k].  Block (q, l), KP threads (k).
__global__ void k_ftc_beta_right(const double* __restrict__ T64, const double* __restrict__ Q,
                                 const size_t* __restrict__ qoff, FtcSpace fs, int N, __half* bA_hi,
                                 __half* bA_lo) {
    const int q = blockIdx.x, l = blockIdx.y, k = threadIdx.x;
    const int j = fs.rj[q], len = FL << j, c0 = fs.ri[q] * len;
    const double* Qj = Q + qoff[j];
    for (int r = 0; r < n_extra(l); ++r) {
        double b = 0.0;
        if (k < l) {
            const double* row = T64 + ((size_t)l * N + r) * N + c0;
            for (int t = 0; t < len; ++t) b = fma(row[t], Qj[(size_t)t * KP + k], b);
        }
        __half h, lo;
        fac_pair(b, h, lo);
        const size_t oa = (((size_t)l * N + r) * fs.FW + q) * KP + k;
        bA_hi[oa] = h;
        bA_lo[oa] = lo;
    }
}

// QT rows of the right intervals: QT[p][(nslots + q, k)][ri len + t] = Q_j[t][k]
// (columns >= 128 carry weight 1).  Block (position over all q, p), KP threads.
__global__ void k_ftc_q_right(const double* __restrict__ Q, const size_t* __restrict__ qoff, FtcSpace fs, int N,
                              __half* qT_hi, __half* qT_lo) {
    int t = blockIdx.x, q = 0;
    while (q + 1 < fs.nright && t >= (FL << fs.rj[q])) {
        t -= FL << fs.rj[q];
        ++q;
    }
    const int j = fs.rj[q], p = blockIdx.y, k = threadIdx.x, c = fs.ri[q] * (FL << j) + t;
    const double v = Q[qoff[j] + (size_t)t * KP + k];
    __half h, lo;
    fac_pair(v, h, lo);
    const size_t ot = (((size_t)p * fs.nslots_f + fs.nslots + q) * KP + k) * N + c;
    qT_hi[ot] = h;
    qT_lo[ot] = lo;
}

// Near band: the diagonal 128 x 128 block of leaf J of T_l,
// D[l][J][r][c] = T_l[128 J + r][128 J + c], and its transpose Dt[l][J][c][r]
// (A operands of the forward rows and the adjoint columns).  Block (J, l).
__global__ void k_ftc_near(const double* __restrict__ T64, int N, __half* D_hi, __half* D_lo, __half* Dt_hi,
                           __half* Dt_lo) {
    const int J = blockIdx.x, l = blockIdx.y, nleaf = N / FL;
    const size_t blk = ((size_t)l * nleaf + J) * FL * FL;
    for (int e = threadIdx.x; e < FL * FL; e += blockDim.x) {
        const int r = e / FL, c = e % FL;
        __half h, lo;
        fac_pair(T64[((size_t)l * N + FL * J + r) * N + FL * J + c], h, lo);
        D_hi[blk + e] = h;
        D_lo[blk + e] = lo;
        Dt_hi[blk + (size_t)c * FL + r] = h;
        Dt_lo[blk + (size_t)c * FL + r] = lo;
    }
}

// Completion block of the adjoint columns: C[l][c][r] = T_l[r][c] for r < 64
// (the completion rows n < n0_l <= 33 and regular rows, which vanish right of
// their diagonal).  Block (column chunk, l).
__global__ void k_ftc_comp(const double* __restrict__ T64, int N, __half* C_hi, __half* C_lo) {
    const int l = blockIdx.y, c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    for (int r = 0; r < BK; ++r) {
        __half h, lo;
        fac_pair(T64[((size_t)l * N + r) * N + c], h, lo);
        C_hi[((size_t)l * N + c) * BK + r] = h;
        C_lo[((size_t)l * N + c) * BK + r] = lo;
    }
}

}  // namespace

struct FtcData {
    FtcSpace base{};   // nleaf, levels, nslots, slot_off
    int np_m = 0, np_w = 0;                        // slot pairs of the MOMENTS / WEIGHTS tiles
    int pa_m[MAX_FSLOTS], pb_m[MAX_FSLOTS], pa_w[MAX_FSLOTS], pb_w[MAX_FSLOTS];
    int NA = 0, NAF = 0;   // augmented widths: adjoint (used slots), forward (+ right slots)
    int lag = kDefaultLag;  // units between a unit's first and second kind in the tile order
    // FP16 pairs (times 2^14): B, BT, QT, QA, the diagonal blocks D and Dt and
    // the completion block C
    __half* bA_hi = nullptr;
    __half* bA_lo = nullptr;
    __half* bT_hi = nullptr;
    __half* bT_lo = nullptr;
    __half* qT_hi = nullptr;
    __half* qT_lo = nullptr;
    __half* qA_hi = nullptr;
    __half* qA_lo = nullptr;
    __half* D_hi = nullptr;
    __half* D_lo = nullptr;
    __half* Dt_hi = nullptr;
    __half* Dt_lo = nullptr;
    __half* C_hi = nullptr;
    __half* C_lo = nullptr;
    CUtensorMap tm_bA_hi, tm_bA_lo, tm_bT_hi, tm_bT_lo, tm_qT_hi, tm_qT_lo, tm_qA_hi, tm_qA_lo;
    CUtensorMap tm_D_hi, tm_D_lo, tm_Dt_hi, tm_Dt_lo, tm_C_hi, tm_C_lo;
};

// MOMENTS / WEIGHTS tiles hold two slots.  Each slot (j, i) of an odd level j
// takes the child slot whose range lies inside its own: (j - 1, 2i) for the
// moments (the interval's columns), (j - 1, 2i + 2) for the adjoint weights
// (the sibling's rows; when that child is a used slot), so the child adds no K
// blocks; a right interval takes its left half, a used slot, the same way; the
// other slots go two by two in order of decreasing length.  Tiles are sorted
// longest first.
static void build_pairs(const FtcSpace& b, int child, bool right, int& npairs, int* pa, int* pb) {
    const int ns = right ? b.nslots_f : b.nslots;
    std::vector<int> taken(ns, 0);
    std::vector<std::pair<int, int>> pairs;
    auto slot = [&](int j, int i) { return b.slot_off[j] + i / 2; };
    for (int j = 1; j < b.levels; j += 2)
        for (int i = 0; i < n_at(b, j); i += 2) {
            if (!used(b, j, i)) continue;
            const int c = 2 * i + child;
            if (!used(b, j - 1, c)) continue;
            pairs.push_back({slot(j, i), slot(j - 1, c)});
            taken[slot(j, i)] = taken[slot(j - 1, c)] = 1;
        }
    if (right)
        for (int q = 0; q < b.nright; ++q) {
            const int j = b.rj[q], i = b.ri[q];
            if (j >= 1 && used(b, j - 1, 2 * i) && !taken[slot(j - 1, 2 * i)]) {
                pairs.push_back({b.nslots + q, slot(j - 1, 2 * i)});
                taken[b.nslots + q] = taken[slot(j - 1, 2 * i)] = 1;
            }
        }
    auto level_of = [&](int s) {
        int j, i;
        slot_ji(b, s, j, i);
        return j;
    };
    std::vector<int> rest;
    for (int s = 0; s < ns; ++s)
        if (!taken[s]) rest.push_back(s);
    std::stable_sort(rest.begin(), rest.end(), [&](int x, int y) { return level_of(x) > level_of(y); });
    for (size_t q = 0; q < rest.size(); q += 2)
        pairs.push_back({rest[q], q + 1 < rest.size() ? rest[q + 1] : -1});
    std::stable_sort(pairs.begin(), pairs.end(), [&](const std::pair<int, int>& x, const std::pair<int, int>& y) {
        return level_of(x.first) > level_of(y.first);
    });
    npairs = (int)pairs.size();
    for (int q = 0; q < npairs; ++q) {
        pa[q] = pairs[q].first;
        pb[q] = pairs[q].second;
    }
}

// The columns [128, N) right of leaf 0 as dyadic intervals (j, i), greedy from
// leaf 1: each the longest interval that starts there on its own alignment and
// ends inside the grid.  For N / 128 = 2^L these are (j, 1), j < L.
static void right_intervals(FtcSpace& b) {
    b.nright = 0;
    for (int p = 1; p < b.nleaf;) {
        int j = 0;
        while ((p % (2 << j)) == 0 && p + (2 << j) <= b.nleaf) ++j;
        b.rj[b.nright] = j;
        b.ri[b.nright] = p >> j;
        ++b.nright;
        p += 1 << j;
    }
}

bool ftc_supported(int N) {
    const int nleaf = N / FL;
    return N % FL == 0 && nleaf >= 2 && nleaf <= (1 << MAX_LEVELS);
}

int ftc_build(dsbt_plan* p, cudaStream_t st) {
    const int N = p->N;
    DSBT_CHECK_ARG(ftc_supported(N), "DSBT_PLAN_FAST_SPLIT needs N a multiple of 128, 256 <= N <= 8192 (N = %d)", N);
    DSBT_CHECK_ARG(p->T64 != nullptr, "DSBT_PLAN_FAST_SPLIT: FP64 factors missing at build");
    FtcData* f = new (std::nothrow) FtcData();
    if (!f) return DSBT_ERR_NOMEM;
    p->ftc = f;
    FtcSpace& b = f->base;
    b.nleaf = N / FL;
    b.levels = 0;
    while ((1 << b.levels) < b.nleaf) ++b.levels;
    b.slot_off[0] = 0;
    for (int j = 0; j < b.levels; ++j) b.slot_off[j + 1] = b.slot_off[j] + n_at(b, j) / 2;   // used slots
    b.nslots = b.slot_off[b.levels];
    right_intervals(b);
    b.nslots_f = b.nslots + b.nright;
    b.FW = std::max(b.levels, b.nright);
    b.KB = N / BK;
    f->NA = b.nslots * KP;
    f->NAF = b.nslots_f * KP;
    build_pairs(b, 0, true, f->np_m, f->pa_m, f->pb_m);
    build_pairs(b, 2, false, f->np_w, f->pa_w, f->pb_w);
    const int levels = b.levels, NA = f->NA, NAF = f->NAF;
    // orthonormal polynomial bases of the levels (host, one thread per level)
    std::vector<std::vector<double>> Qh(levels);
    std::vector<std::thread> pool;
    for (int j = 0; j < levels; ++j) pool.emplace_back([&, j]() { poly_basis(FL << j, Qh[j]); });
    for (auto& t : pool) t.join();
    std::vector<size_t> qoff(levels);
    size_t qtot = 0;
    for (int j = 0; j < levels; ++j) {
        qoff[j] = qtot;
        qtot += Qh[j].size();
    }
    std::vector<double> Qall(qtot);
    for (int j = 0; j < levels; ++j) std::copy(Qh[j].begin(), Qh[j].end(), Qall.begin() + qoff[j]);
    const size_t L = (size_t)p->l_max + 1;
    // compact B [l][r][FW][64] and BT [l][levels][64][N]; dense QT [2][NAF][N] and QA [2][N][NA]
    const size_t nbA = L * N * b.FW * KP, nbT = L * b.levels * KP * N, nqT = 2 * (size_t)N * NAF,
                 nq = 2 * (size_t)N * NA;
    const size_t nD = L * N * FL, nC = L * N * BK;
    const size_t hb = sizeof(__half);
    double* Qd = nullptr;
    size_t* qoffd = nullptr;
    bool ok = cudaMalloc((void**)&f->bA_hi, nbA * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->bA_lo, nbA * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->bT_hi, nbT * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->bT_lo, nbT * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->qT_hi, nqT * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->qT_lo, nqT * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->qA_hi, nq * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->qA_lo, nq * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->D_hi, nD * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->D_lo, nD * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->Dt_hi, nD * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->Dt_lo, nD * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->C_hi, nC * hb) == cudaSuccess &&
              cudaMalloc((void**)&f->C_lo, nC * hb) == cudaSuccess &&
              cudaMalloc((void**)&Qd, qtot * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&qoffd, levels * sizeof(size_t)) == cudaSuccess;
    ok = ok && cudaMemcpy(Qd, Qall.data(), qtot * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(qoffd, qoff.data(), levels * sizeof(size_t), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(Qd);
        cudaFree(qoffd);
        set_error("DSBT_PLAN_FAST_SPLIT: device allocation or copy failed");
        return DSBT_ERR_NOMEM;
    }
    for (__half* a : {f->bA_hi, f->bA_lo}) DSBT_CUDA_TRY(cudaMemsetAsync(a, 0, nbA * hb, st));
    for (__half* a : {f->bT_hi, f->bT_lo}) DSBT_CUDA_TRY(cudaMemsetAsync(a, 0, nbT * hb, st));
    for (__half* a : {f->qT_hi, f->qT_lo}) DSBT_CUDA_TRY(cudaMemsetAsync(a, 0, nqT * hb, st));
    for (__half* a : {f->qA_hi, f->qA_lo}) DSBT_CUDA_TRY(cudaMemsetAsync(a, 0, nq * hb, st));
    {
        ProfScope ps(kKPlan, st);
        k_ftc_beta<<<dim3(levels * N, (unsigned)L), KP, 0, st>>>(p->T64, Qd, qoffd, b, N, f->bA_hi, f->bA_lo,
                                                                       f->bT_hi, f->bT_lo);
        k_ftc_q<<<dim3(levels * N, 2), KP, 0, st>>>(Qd, qoffd, b, N, f->qT_hi, f->qT_lo, f->qA_hi, f->qA_lo);
        k_ftc_beta_right<<<dim3(b.nright, (unsigned)L), KP, 0, st>>>(p->T64, Qd, qoffd, b, N, f->bA_hi, f->bA_lo);
        k_ftc_q_right<<<dim3(N - FL, 2), KP, 0, st>>>(Qd, qoffd, b, N, f->qT_hi, f->qT_lo);
        k_ftc_near<<<dim3(b.nleaf, (unsigned)L), 256, 0, st>>>(p->T64, N, f->D_hi, f->D_lo, f->Dt_hi, f->Dt_lo);
        k_ftc_comp<<<dim3((N + 255) / 256, (unsigned)L), 256, 0, st>>>(p->T64, N, f->C_hi, f->C_lo);
    }
    DSBT_CUDA_TRY(cudaGetLastError());
    DSBT_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(Qd);
    cudaFree(qoffd);
    int rc = encode_tmap_f16_sw128(&f->tm_bA_hi, f->bA_hi, L * N, (uint64_t)b.FW * KP, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_bA_lo, f->bA_lo, L * N, (uint64_t)b.FW * KP, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_bT_hi, f->bT_hi, L * levels * KP, N, 64, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_bT_lo, f->bT_lo, L * levels * KP, N, 64, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_qT_hi, f->qT_hi, 2 * (uint64_t)NAF, N, 64, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_qT_lo, f->qT_lo, 2 * (uint64_t)NAF, N, 64, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_qA_hi, f->qA_hi, 2 * (uint64_t)N, NA, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_qA_lo, f->qA_lo, 2 * (uint64_t)N, NA, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_D_hi, f->D_hi, L * N, FL, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_D_lo, f->D_lo, L * N, FL, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_Dt_hi, f->Dt_hi, L * N, FL, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_Dt_lo, f->Dt_lo, L * N, FL, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_C_hi, f->C_hi, L * N, BK, 128, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&f->tm_C_lo, f->C_lo, L * N, BK, 128, BK);
    return rc;
}

void ftc_free(dsbt_plan* p) {
    if (!p || !p->ftc) return;
    FtcData* f = p->ftc;
    for (__half* a : {f->bA_hi, f->bA_lo, f->bT_hi, f->bT_lo, f->qT_hi, f->qT_lo, f->qA_hi, f->qA_lo, f->D_hi,
                      f->D_lo, f->Dt_hi, f->Dt_lo, f->C_hi, f->C_lo})
        cudaFree(a);
    delete f;
    p->ftc = nullptr;
}

// Augmented lines (an FP16 pair of NAF values per line), then the counter
// block of a launch: scheduler, abort word and one counter per unit (a unit
// is a column tile of BN_MAX lines of one group).
static size_t ftc_aug_bytes(const dsbt_plan* p, size_t lines) {
    return (2 * lines * (size_t)p->ftc->NAF * sizeof(__half) + 255) & ~(size_t)255;
}

size_t ftc_scratch_bytes(const dsbt_plan* p, size_t lines) {
    if (!p->ftc) return 0;
    return ftc_aug_bytes(p, lines) + sizeof(int) * (kCtrUnits + lines / BN_MAX + kMaxGroups + 1);
}

void ftc_set_lag(dsbt_plan* p, int lag) {
    if (p->ftc) p->ftc->lag = lag;
}

namespace {

// One launch over the groups (largest l first): the first kind (MOMENTS or
// WEIGHTS) and the second (EVAL or LEAFOUT) of every unit, interleaved.
int launch_fused(const dsbt_plan* p, const GroupTable& g, int dir, const CUtensorMap& a0h, const CUtensorMap& a0l,
                 const CUtensorMap& a1h, const CUtensorMap& a1l, const CUtensorMap& b1h, const CUtensorMap& b1l,
                 const CUtensorMap& a2h, const CUtensorMap& a2l, const CUtensorMap& b2h, const CUtensorMap& b2l,
                 const CUtensorMap& a3h, const CUtensorMap& a3l, const EpiArgs& ep, int* ctr, size_t lines,
                 cudaStream_t st) {
    const FtcData* f = p->ftc;
    FtcSpace fs = f->base;
    const bool fwd = dir > 0;
    fs.amode = fwd ? kMoments : kWeights;
    fs.omode = fwd ? kEval : kLeafOut;
    fs.kc = KC;
    // first row past the A table of the tile's slots (QT or the compact BT)
    fs.a_oob = fwd ? 2 * fs.nslots_f * KP : (p->l_max + 1) * fs.levels * KP;
    fs.npairs = fwd ? f->np_m : f->np_w;
    for (int q = 0; q < fs.npairs; ++q) {
        fs.pair_a[q] = fwd ? f->pa_m[q] : f->pa_w[q];
        fs.pair_b[q] = fwd ? f->pb_m[q] : f->pb_w[q];
    }
    fs.RT = p->N / BM;
    fs.npos = g.ngroups;
    fs.u0[0] = 0;
    fs.acum[0] = 0;
    for (int i = 0; i < g.ngroups; ++i) {
        const int gi = g.ngroups - 1 - i;
        const int nl = g.line0[gi + 1] - g.line0[gi];
        fs.order[i] = gi;
        const int ct = (nl + BN_MAX - 1) / BN_MAX;
        fs.ta[i] = g.l[gi] == 0 ? 0 : fs.npairs;   // T_0 has no entries left of its diagonal
        fs.u0[i + 1] = fs.u0[i] + ct;
        fs.acum[i + 1] = fs.acum[i] + ct * fs.ta[i];
    }
    fs.units = fs.u0[g.ngroups];
    if (fs.units == 0) return DSBT_OK;
    if ((size_t)fs.units > lines / BN_MAX + kMaxGroups + 1) {
        set_error("interval-scheme contraction: unit counters exceed the scratch");
        return DSBT_ERR_INVALID;
    }
    fs.lag = std::max(1, std::min(f->lag, fs.units));
    fs.total = fs.acum[g.ngroups] + fs.units * fs.RT;
    const size_t smem = (size_t)STAGES * STAGE_BYTES + 1024 + 512;
    int rc = ensure_smem((const void*)k_contract_ftc, smem);
    if (rc) return rc;
    int dev = 0, nsm = 0;
    DSBT_CUDA_TRY(cudaGetDevice(&dev));
    DSBT_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const int grid = fs.total < nsm ? fs.total : nsm;
    DSBT_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(int) * (kCtrUnits + fs.units), st));
    ProfScope ps(kKContractTF32, st);
    k_contract_ftc<<<grid, NTHREADS, smem, st>>>(a0h, a0l, a1h, a1l, b1h, b1l, a2h, a2l, b2h, b2l, a3h, a3l, g, fs,
                                                 p->N, ep, p->status, p->spin_limit, ctr);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

}  // namespace

int contract_split_fast(const dsbt_plan* p, const GroupTable& g, int dir, const __half* in_hi, const __half* in_lo,
                        const float* scale, int out_mode, void* out0, void* out1, const float2* phase, void* scratch,
                        cudaStream_t st) {
    const FtcData* f = p->ftc;
    if (!f) {
        set_error("interval-scheme contraction needs a plan built with DSBT_PLAN_FAST_SPLIT");
        return DSBT_ERR_UNSUPPORTED;
    }
    if (g.total_lines == 0) return DSBT_OK;
    if (out_mode == kOutPlanarSplit || out_mode == kOutUserC64) {
        for (int i = 0; i < g.ngroups; ++i) {
            if ((g.line0[i] & 1) || ((g.line0[i + 1] - g.line0[i]) & 1)) {
                set_error("complex output needs whole channels per group");
                return DSBT_ERR_INVALID;
            }
        }
    }
    const int N = p->N, NA = dir > 0 ? f->NAF : f->NA;   // augmented width of this direction
    const size_t R = (size_t)g.total_lines;
    __half* aug_hi = reinterpret_cast<__half*>(scratch);
    __half* aug_lo = aug_hi + R * NA;
    int* ctr = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(scratch) + ftc_aug_bytes(p, R));
    CUtensorMap in_h, in_l, aug_h, aug_l;
    int rc = encode_tmap_f16_sw128(&in_h, in_hi, R, N, BBOX, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&in_l, in_lo, R, N, BBOX, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&aug_h, aug_hi, R, NA, BBOX, BK);
    if (rc == DSBT_OK) rc = encode_tmap_f16_sw128(&aug_l, aug_lo, R, NA, BBOX, BK);
    if (rc != DSBT_OK) return rc;
    const EpiArgs ep{out_mode, out0, out1, phase, p->knl != nullptr, scale, aug_hi, aug_lo, NA};
    if (dir > 0)
        return launch_fused(p, g, dir, f->tm_qT_hi, f->tm_qT_lo, f->tm_D_hi, f->tm_D_lo, in_h, in_l, f->tm_bA_hi,
                            f->tm_bA_lo, aug_h, aug_l, f->tm_D_hi, f->tm_D_lo, ep, ctr, R, st);
    return launch_fused(p, g, dir, f->tm_bT_hi, f->tm_bT_lo, f->tm_Dt_hi, f->tm_Dt_lo, in_h, in_l, f->tm_qA_hi,
                        f->tm_qA_lo, aug_h, aug_l, f->tm_C_hi, f->tm_C_lo, ep, ctr, R, st);
}

}  // namespace dsbt
