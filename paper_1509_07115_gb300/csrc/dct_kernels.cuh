// dct_kernels.cuh -- the batched sine / cosine transform kernels (templates),
// shared by dct.cu (FP64 and TF32-split instantiations) and dct_f32.cu (the
// FP32 kernels of the split-FP16 path, one instantiation per plan grid).
//
// F_l (Sec. 2.2, Eq. (16)) is the orthonormal DCT-II for odd l and the
// orthonormal DST-II for even l on the midpoint grid r_i = (i - 1/2) dr.  The
// DST-II reduces to the DCT-II of (-1)^i psi_i read backwards:
//     f_{N-k} = DCT-II((-1)^i psi)_k,   i.e. storage index n - 1 = N - 1 - k.
// Each DCT-II of length N is computed with one complex FFT of length N after
// the even/odd reordering v_j = x_{2j}, v_{N-1-j} = x_{2j+1}:
//     X_k = 1/2 [w_k V_k + conj(w_k) V_{(N-k) mod N}],  w_k = exp(-i pi k / (2N)),
// which holds for complex x as well, so one complex channel (two real lines)
// costs one FFT.  The transpose F_l^T (DCT-III) inverts those steps:
//     V_k = conj(w_k) (X_k - i X_{N-k}) (X_N = 0),  v = IFFT(V),  x_{2j} = v_j,
//     x_{2j+1} = v_{N-1-j}.
//
// FFT: Stockham autosort in shared memory for N = 256 q (q = 1..32): radix-16
// stages (16 values per thread in registers, a 4 x 4 register DFT), one
// radix-2/4/8 stage, then one direct radix-Q stage for the odd part Q of q
// (kernels are instantiated per Q), with
// N/16 threads per line and several lines per CTA when N/16 < 256.  Shared
// memory is padded by one element every 16, which makes every stage's loads
// and stores free of bank conflicts.  Twiddles of a radix-16 butterfly come
// from two table loads (w, w^4) and products of depth <= 3.  The forward
// transform's global loads move two complex values per thread (16 or 32
// bytes), the pair (x_{2j}, x_{2j+1}) that the reordering sends to v_j and
// v_{N-1-j}, through shared memory; the inverse runs its first radix-16 stage
// on the V_k it has just formed in registers.  (Loading each thread's first
// butterfly inputs straight from global memory in the forward transform made
// it slower: the stride-2 loads cost more than the shared-memory pass.)
// A kernel is instantiated either per Q with N at run time (NS = 0) or with N
// fixed at compile time (NS = N): every padded shared-memory index is then
// one base per thread plus constant offsets (all index steps are multiples of
// 16), which removes most of the integer work of the stages.  The FP32 kernels
// of the split-FP16 path have one instantiation per plan grid; the FP64 and
// TF32-split kernels for N = 2048, 4096, 8192 and per Q otherwise.
#pragma once

#include <cuda_fp16.h>

#include "plan.cuh"

namespace dsbt {


template <typename R> struct Cx;
template <> struct Cx<float> { typedef float2 T; };
template <> struct Cx<double> { typedef double2 T; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {   // a * conj(b)
    C r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename C> __device__ __forceinline__ C cmi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }  // -i a

template <typename C> __device__ __forceinline__ void dft2(C& a, C& b) { C t = a; a = cadd(t, b); b = csub(t, b); }

template <typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
    C s02 = cadd(x0, x2), d02 = csub(x0, x2), s13 = cadd(x1, x3), d13 = cmi(csub(x1, x3));
    x0 = cadd(s02, s13);
    x2 = csub(s02, s13);
    x1 = cadd(d02, d13);
    x3 = csub(d02, d13);
}

template <typename C> __device__ __forceinline__ void dft8(C* x) {
    typedef decltype(x[0].x) R;
    const R h = (R)0.70710678118654752440;
    C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6];
    C o0 = x[1], o1 = x[3], o2 = x[5], o3 = x[7];
    dft4(e0, e1, e2, e3);
    dft4(o0, o1, o2, o3);
    C t1; t1.x = h * (o1.x + o1.y); t1.y = h * (o1.y - o1.x);     // exp(-i pi/4) o1
    C t2 = cmi(o2);                                               // -i o2
    C t3; t3.x = h * (o3.y - o3.x); t3.y = -h * (o3.x + o3.y);    // exp(-3 i pi/4) o3
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, t1); x[5] = csub(e1, t1);
    x[2] = cadd(e2, t2); x[6] = csub(e2, t2);
    x[3] = cadd(e3, t3); x[7] = csub(e3, t3);
}

// 16-point DFT as 4 x 4: X[k1 + 4 k2] = sum_n2 W4^{n2 k2} W16^{n2 k1} sum_n1 x[4 n1 + n2] W4^{n1 k1}.
template <typename C> __device__ __forceinline__ void dft16(C* x) {
    typedef decltype(x[0].x) R;
    const R c8 = (R)0.92387953251128675613, s8 = (R)0.38268343236508977173, h = (R)0.70710678118654752440;
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft4(x[n2], x[4 + n2], x[8 + n2], x[12 + n2]);
    // x[4 k1 + n2] holds A[n2][k1]; multiply by W16^{n2 k1}
    C t;
    t = x[5];  x[5].x = c8 * t.x + s8 * t.y;  x[5].y = c8 * t.y - s8 * t.x;     // W^1
    t = x[6];  x[6].x = h * (t.x + t.y);       x[6].y = h * (t.y - t.x);         // W^2
    t = x[7];  x[7].x = s8 * t.x + c8 * t.y;  x[7].y = s8 * t.y - c8 * t.x;     // W^3
    t = x[9];  x[9].x = h * (t.x + t.y);       x[9].y = h * (t.y - t.x);         // W^2
    x[10] = cmi(x[10]);                                                          // W^4
    t = x[11]; x[11].x = h * (t.y - t.x);      x[11].y = -h * (t.x + t.y);      // W^6
    t = x[13]; x[13].x = s8 * t.x + c8 * t.y; x[13].y = s8 * t.y - c8 * t.x;    // W^3
    t = x[14]; x[14].x = h * (t.y - t.x);      x[14].y = -h * (t.x + t.y);      // W^6
    t = x[15]; x[15].x = -c8 * t.x - s8 * t.y; x[15].y = s8 * t.x - c8 * t.y;  // W^9
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) dft4(x[4 * k1], x[4 * k1 + 1], x[4 * k1 + 2], x[4 * k1 + 3]);
    // x[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4 x 4 block
    C y[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
    for (int i = 0; i < 16; ++i) x[i] = y[i];
}

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }

// Padded distance of two elements d apart, for d a multiple of 16: padi(i + d)
// = padi(i) + pstride(d) for every i >= 0 (and padi(i - d) = padi(i) -
// pstride(d) for i >= d).  Every distance the transforms step by is a multiple
// of 16 (N = 256 q), so each thread forms one padded base index and adds
// multiples of a stride that is a compile-time constant when N is.
__device__ __forceinline__ int pstride(int d) { return d + (d >> 4); }

// One Stockham stage of radix RX on one line's padded shared buffer s; the
// line has T = N/16 threads (lt = thread index within the line), each owning
// 16/RX butterflies.  Barriers are CTA-wide (all lines run the same stages).
template <int RX, int NS, typename C>
__device__ __forceinline__ void stockham_stage(C* s, const C* __restrict__ tw, int N, int Ls, int lt, int T) {
    constexpr int PER = 16 / RX;
    const int nb = N / RX;
    const int sn = pstride(nb);
    C x[PER][RX];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = lt + u * T;
        const int k = j & (Ls - 1);
        const int b = k * (N / (Ls * RX));     // twiddle w = W_N^b, factor r uses w^r
        if (NS > 0) {   // constant strides from one padded base
            const C* src = s + padi(j);
#pragma unroll
            for (int r = 0; r < RX; ++r) x[u][r] = src[r * sn];
        } else {        // fewer live registers for run-time N
#pragma unroll
            for (int r = 0; r < RX; ++r) x[u][r] = s[padi(j + r * nb)];
        }
        if (k > 0) {
            if (RX == 16) {
                const C w1 = tw[b], w4 = tw[4 * b];
                const C w2 = cmul(w1, w1), w3 = cmul(w2, w1), w8 = cmul(w4, w4), w12 = cmul(w8, w4);
                const C lo[4] = {w1, w1, w2, w3};
                const C hi[4] = {w4, w4, w8, w12};
#pragma unroll
                for (int r = 1; r < 16; ++r) {
                    const int a = r & 3, c = r >> 2;
                    C w;
                    if (c == 0) w = lo[a];
                    else if (a == 0) w = hi[c];
                    else w = cmul(hi[c], lo[a]);
                    x[u][r] = cmul(x[u][r], w);
                }
            } else {
#pragma unroll
                for (int r = 1; r < RX; ++r) x[u][r] = cmul(x[u][r], tw[r * b]);
            }
        }
        if (RX == 16) dft16(x[u]);
        else if (RX == 8) dft8(x[u]);
        else if (RX == 4) dft4(x[u][0], x[u][1], x[u][2], x[u][3]);
        else dft2(x[u][0], x[u][1]);
    }
    __syncthreads();
    // outputs base + q Ls: Ls is 1 only in the first stage (radix 16, base a
    // multiple of 16, so the 16 outputs share one padded row), else a multiple of 16
    const int sl = Ls == 1 ? 1 : pstride(Ls);
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = lt + u * T;
        const int k = j & (Ls - 1);
        const int base = (j - k) * RX + k;
        if (NS > 0) {
            C* dst = s + padi(base);
#pragma unroll
            for (int q = 0; q < RX; ++q) dst[q * sl] = x[u][q];
        } else {
#pragma unroll
            for (int q = 0; q < RX; ++q) s[padi(base + q * Ls)] = x[u][q];
        }
    }
    __syncthreads();
}

template <typename C> struct Re;
template <> struct Re<float2> { typedef float T; };
template <> struct Re<double2> { typedef double T; };

// The last Stockham stage for N = 256 q: radix Q = the odd part of q (3..31,
// prime or not), a direct DFT per butterfly.  In the last stage (Ls = N/Q)
// butterfly j reads and writes the same Q elements j + r N/Q, so each thread
// finishes one butterfly before the next without a barrier in between.
// Inputs are paired, S_r = y_r + y_{Q-r} and D_r = y_r - y_{Q-r}, so outputs q
// and Q - q share one pass: X_q = A - iB, X_{Q-q} = A + iB with
// A = y_0 + sum_r S_r cos(2 pi r q / Q), B = sum_r D_r sin(2 pi r q / Q).
// The Q-th roots of unity come from shared memory (sroot[m] = exp(-2 pi i m / Q),
// filled by the caller).
template <int Q, typename C>
__device__ __forceinline__ void stockham_last_odd(C* s, const C* __restrict__ tw, const C* sroot, int N,
                                                  int lt, int T) {
    typedef typename Re<C>::T R;
    constexpr int H = (Q - 1) / 2;
    const int nb = N / Q;          // 256 q / Q: a multiple of 16
    const int sn = pstride(nb);
    for (int j = lt; j < nb; j += T) {
        C* row = s + padi(j);
        C y0, S[H], D[H];
        {
            C x[Q];
#pragma unroll
            for (int r = 0; r < Q; ++r) x[r] = row[r * sn];
            if (j > 0) {
#pragma unroll
                for (int r = 1; r < Q; ++r) x[r] = cmul(x[r], tw[r * j]);
            }
            y0 = x[0];
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                S[r - 1] = cadd(x[r], x[Q - r]);
                D[r - 1] = csub(x[r], x[Q - r]);
            }
        }
        C X0 = y0;
#pragma unroll
        for (int r = 0; r < H; ++r) X0 = cadd(X0, S[r]);
        row[0] = X0;
#pragma unroll 1
        for (int q = 1; q <= H; ++q) {
            C A = y0, B;
            B.x = B.y = (R)0;
            int e = 0;
#pragma unroll
            for (int r = 1; r <= H; ++r) {
                e += q;
                if (e >= Q) e -= Q;   // e = r q mod Q
                const C w = sroot[e];
                const R c = w.x, sn = -w.y;
                A.x += S[r - 1].x * c;
                A.y += S[r - 1].y * c;
                B.x += D[r - 1].x * sn;
                B.y += D[r - 1].y * sn;
            }
            C Xq, Xm;
            Xq.x = A.x + B.y;
            Xq.y = A.y - B.x;
            Xm.x = A.x - B.y;
            Xm.y = A.y + B.x;
            row[q * sn] = Xq;
            row[(Q - q) * sn] = Xm;
        }
    }
    __syncthreads();
}

// Forward FFT of length N = 256 q, q = 2^a Q: radix-16 stages, one radix-2/4/8
// stage for the rest of the power of two and, when Q > 1, one radix-Q stage
// (sroot is a 32-entry shared scratch for its roots).
template <int Q, int NS, typename C>
__device__ __forceinline__ void fft_stages(C* s, const C* __restrict__ tw, C* sroot, int N, int lt, int T, int Ls,
                                           int rem) {
    while ((rem & 15) == 0) {
        stockham_stage<16, NS>(s, tw, N, Ls, lt, T);
        Ls *= 16;
        rem >>= 4;
    }
    if ((rem & 7) == 0) { stockham_stage<8, NS>(s, tw, N, Ls, lt, T); Ls *= 8; rem >>= 3; }
    else if ((rem & 3) == 0) { stockham_stage<4, NS>(s, tw, N, Ls, lt, T); Ls *= 4; rem >>= 2; }
    else if ((rem & 1) == 0) { stockham_stage<2, NS>(s, tw, N, Ls, lt, T); Ls *= 2; rem >>= 1; }
    if constexpr (Q > 1) {
        for (int m = threadIdx.x; m < Q; m += blockDim.x) sroot[m] = tw[m * (N / Q)];   // W_Q^m
        __syncthreads();
        stockham_last_odd<Q>(s, tw, sroot, N, lt, T);   // Ls = N / Q here
    }
}

// Forward FFT of length N = 256 q whose input is already in registers:
// x[r] = element lt + r T of the line (T = N/16), i.e. exactly the inputs of
// butterfly lt of the first radix-16 Stockham stage (Ls = 1, no twiddles).
// That stage runs on the registers and writes its outputs 16 lt + q to the
// line's shared buffer s, then the remaining stages follow (fft_stages).
// The caller must have finished every read of s before the call.
template <int Q, int NS, typename C>
__device__ __forceinline__ void fft_from_registers(C* s, C* x, const C* __restrict__ tw, C* sroot, int N, int lt,
                                                   int T) {
    dft16(x);
    C* dst = s + 17 * lt;   // padi(16 lt + q) for q < 16
#pragma unroll
    for (int q = 0; q < 16; ++q) dst[q] = x[q];
    __syncthreads();
    fft_stages<Q, NS>(s, tw, sroot, N, lt, T, 16, N >> 4);
}

__device__ __forceinline__ int find_group(const GroupTable& g, int chan) {
    int lo = 0, hi = g.ngroups - 1;
    while (lo < hi) {   // last group with chan0 <= chan
        const int mid = (lo + hi + 1) >> 1;
        if (g.chan0[mid] <= chan) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <typename C> __device__ __forceinline__ void ld_pair(const C* p, C& a, C& b);
template <> __device__ __forceinline__ void ld_pair<float2>(const float2* p, float2& a, float2& b) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
template <> __device__ __forceinline__ void ld_pair<double2>(const double2* p, double2& a, double2& b) {
    a = p[0];
    b = p[1];
}
__device__ __forceinline__ void ld_real_pair(const float* p, float& a, float& b) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
}
__device__ __forceinline__ void ld_real_pair(const double* p, double& a, double& b) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
}
template <typename C> __device__ __forceinline__ void st_pair(C* p, C a, C b);
template <> __device__ __forceinline__ void st_pair<float2>(float2* p, float2 a, float2 b) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
template <> __device__ __forceinline__ void st_pair<double2>(double2* p, double2 a, double2 b) {
    p[0] = a;
    p[1] = b;
}

// Lines per CTA: as many lines of N/16 threads as fit in 256 threads (one
// line of up to 512 threads when N/16 > 256).
__host__ __device__ inline int lines_per_cta(int N) { return (N / 16 >= 256) ? 1 : 256 / (N / 16); }

// Output modes of the forward transform (planar lines, storage index n - p_l):
// kPlain: R values; kSplitTF32: the TF32 pair hi + lo as two FP32 lines;
// kSplitF16: the channel scaled by a power of two 2^e with ||2^e psi|| in
// [2^12, 2^13), then the FP16 pair hi = fp16(v), lo = fp16(v - hi), and the
// unscale factor 2^-e per line in `scale`.  FP16 keeps 11 significant bits
// like TF32; the scale keeps every value of the orthogonal transforms that
// follow far below the FP16 range (|v| <= ||v|| < 2^13.5) and puts the FP16
// subnormal step (2^-24) 2^-36 below the channel norm.
enum : int { kPlain = 0, kSplitTF32 = 1, kSplitF16 = 2 };

// Power-of-two exponent e with x 2^e in [2^12, 2^13) (0 for 0, inf, nan).
__device__ __forceinline__ int scale_exp(float nrm) {
    return (nrm > 0.f && isfinite(nrm)) ? 12 - ilogbf(nrm) : 0;
}

// Forward transform.  FP32 kernels: at most 64 registers, so two CTAs of
// up to 512 threads (one line of N/16 threads each) fit on an SM.  NS > 0 is
// the grid size fixed at compile time (every index step a constant), NS = 0
// takes N at run time.
template <typename R, int MODE, int Q, int NS>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1) k_dct_fwd(GroupTable g, int Nrt, int cplx, const R* __restrict__ in,
                                                 void* __restrict__ out0, void* __restrict__ out1,
                                                 float* __restrict__ scale,
                                                 const typename Cx<R>::T* __restrict__ tw,
                                                 const typename Cx<R>::T* __restrict__ post) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ float spart[32];   // per 16 threads (<= 512 threads): partial sums of |psi_i|^2
    const int N = NS ? NS : Nrt;
    const int T = N >> 4;
    const int G = lines_per_cta(N);
    const int grp = threadIdx.x / T, lt = threadIdx.x % T;
    C* s = reinterpret_cast<C*>(smem_raw) + (size_t)grp * (N + (N >> 4));
    const int chan = blockIdx.x * G + grp;
    const int nchan = g.chan0[g.ngroups];
    const bool live = chan < nchan;
    int gi = 0, l = 0, local = 0;
    if (live) {
        gi = find_group(g, chan);
        l = g.l[gi];
        local = chan - g.chan0[gi];
    }
    const bool even = (l & 1) == 0;
    const size_t ubase = !live ? 0 : (g.uoff ? (size_t)g.uoff[chan] : (size_t)chan * N);   // caller's element offset
    // load pairs (x_{2j}, x_{2j+1}) -> v_j, v_{N-1-j}; all loads issued before the stores
    C a[8], b[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int j = lt + u * T;
        if (!live) {
            a[u].x = a[u].y = b[u].x = b[u].y = (R)0;
        } else if (cplx) {
            ld_pair(reinterpret_cast<const C*>(in) + ubase + 2 * j, a[u], b[u]);
        } else {
            a[u].x = in[ubase + 2 * j];
            b[u].x = in[ubase + 2 * j + 1];
            a[u].y = b[u].y = (R)0;
        }
    }
    float part = 0.f;
    if (MODE == kSplitF16) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
            part += (float)(a[u].x * a[u].x + a[u].y * a[u].y) + (float)(b[u].x * b[u].x + b[u].y * b[u].y);
    }
    {
        C* lo = s + padi(lt);            // v_j, j = lt + u T
        C* hi = s + padi(N - 1 - lt);    // v_{N-1-j}
        const int st = pstride(T);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (even) { b[u].x = -b[u].x; b[u].y = -b[u].y; }
            if (NS > 0) {
                lo[u * st] = a[u];
                hi[-u * st] = b[u];
            } else {
                const int j = lt + u * T;
                s[padi(j)] = a[u];
                s[padi(N - 1 - j)] = b[u];
            }
        }
    }
    __syncthreads();
    if (MODE == kSplitF16) {
        // sum over the line's T threads (T a multiple of 16) in a fixed order, so
        // that the scale never depends on timing: 16-lane groups by shuffles, one
        // shared slot per group, summed in slot order below (the FFT's barriers
        // order the slots before those reads).  blockDim is a multiple of 16, so
        // a warp is 32 or (the last one) 16 threads.
        const unsigned mask = (blockDim.x - (threadIdx.x & ~31u)) >= 32 ? 0xffffffffu : 0x0000ffffu;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(mask, part, o);
        if ((threadIdx.x & 15) == 0) spart[threadIdx.x >> 4] = part;
    }
    __shared__ C sroot[32];
    fft_stages<Q, NS>(s, tw, sroot, N, lt, T, 1, N);
    if (!live) return;
    const R sc1 = (R)sqrt(2.0 / (double)N), sc0 = (R)sqrt(1.0 / (double)N);
    const int line = g.line0[gi] + (cplx ? 2 * local : local);
    float fs = 1.f;
    if (MODE == kSplitF16) {
        float nrm2 = 0.f;
        for (int q = grp * (T >> 4); q < (grp + 1) * (T >> 4); ++q) nrm2 += spart[q];
        const int e = scale_exp(sqrtf(nrm2));
        fs = ldexpf(1.f, e);
        if (lt == 0) {
            scale[line] = ldexpf(1.f, -e);
            if (cplx) scale[line + 1] = ldexpf(1.f, -e);
        }
    }
    const int st2 = pstride(2 * T);
#pragma unroll
    for (int i = 0; i < 8; ++i) {   // m = lt + i T, N / 2 = 8 T
        const int m = lt + i * T;
        C X[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int k = 2 * m + e;
            // V_k and V_{N-k} (V_0 for k = 0)
            const C a = NS > 0 ? s[padi(2 * lt + e) + i * st2] : s[padi(k)];
            const C b = (k == 0) ? a : (NS > 0 ? s[padi(N - 2 * lt - e) - i * st2] : s[padi(N - k)]);
            const C w = post[k];
            C v;   // 1/2 (w a + conj(w) b)
            v.x = (R)0.5 * ((w.x * a.x - w.y * a.y) + (w.x * b.x + w.y * b.y));
            v.y = (R)0.5 * ((w.x * a.y + w.y * a.x) + (w.x * b.y - w.y * b.x));
            const R sc = (k == 0) ? sc0 : sc1;
            v.x *= sc;
            v.y *= sc;
            X[e] = v;
        }
        // storage index of k: odd l -> k; even l -> N-1-k (pairs stay adjacent, order flips)
        const int idx = even ? (N - 2 - 2 * m) : 2 * m;
        const C lo_e = even ? X[1] : X[0], hi_e = even ? X[0] : X[1];   // elements at idx, idx+1
        if (MODE == kSplitTF32) {
            float* o0 = reinterpret_cast<float*>(out0) + (size_t)line * N;
            float* o1 = reinterpret_cast<float*>(out1) + (size_t)line * N;
            const float r0 = round_tf32((float)lo_e.x), r1 = round_tf32((float)hi_e.x);
            *reinterpret_cast<float2*>(o0 + idx) = make_float2(r0, r1);
            *reinterpret_cast<float2*>(o1 + idx) =
                make_float2(round_tf32((float)lo_e.x - r0), round_tf32((float)hi_e.x - r1));
            if (cplx) {
                const float i0 = round_tf32((float)lo_e.y), i1 = round_tf32((float)hi_e.y);
                *reinterpret_cast<float2*>(o0 + N + idx) = make_float2(i0, i1);
                *reinterpret_cast<float2*>(o1 + N + idx) =
                    make_float2(round_tf32((float)lo_e.y - i0), round_tf32((float)hi_e.y - i1));
            }
        } else if (MODE == kSplitF16) {
            __half* o0 = reinterpret_cast<__half*>(out0) + (size_t)line * N;
            __half* o1 = reinterpret_cast<__half*>(out1) + (size_t)line * N;
            const float2 vr = make_float2((float)lo_e.x * fs, (float)hi_e.x * fs);
            const __half2 hr = __float22half2_rn(vr);
            *reinterpret_cast<__half2*>(o0 + idx) = hr;
            *reinterpret_cast<__half2*>(o1 + idx) = __float22half2_rn(
                make_float2(vr.x - __low2float(hr), vr.y - __high2float(hr)));
            if (cplx) {
                const float2 vi = make_float2((float)lo_e.y * fs, (float)hi_e.y * fs);
                const __half2 hi2 = __float22half2_rn(vi);
                *reinterpret_cast<__half2*>(o0 + N + idx) = hi2;
                *reinterpret_cast<__half2*>(o1 + N + idx) = __float22half2_rn(
                    make_float2(vi.x - __low2float(hi2), vi.y - __high2float(hi2)));
            }
        } else {
            R* o0 = reinterpret_cast<R*>(out0) + (size_t)line * N;
            o0[idx] = lo_e.x;
            o0[idx + 1] = hi_e.x;
            if (cplx) {
                o0[N + idx] = lo_e.y;
                o0[N + idx + 1] = hi_e.y;
            }
        }
    }
}

// Inverse transform F_l^T: planar lines -> caller layout (NS as in k_dct_fwd).
template <typename R, int Q, int NS>
__global__ void __launch_bounds__(512, sizeof(R) == 4 ? 2 : 1) k_dct_inv(GroupTable g, int Nrt, int cplx, const R* __restrict__ in,
                                                 R* __restrict__ out, const typename Cx<R>::T* __restrict__ tw,
                                                 const typename Cx<R>::T* __restrict__ post) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int N = NS ? NS : Nrt;
    const int T = N >> 4;
    const int G = lines_per_cta(N);
    const int grp = threadIdx.x / T, lt = threadIdx.x % T;
    C* s = reinterpret_cast<C*>(smem_raw) + (size_t)grp * (N + (N >> 4));
    const int chan = blockIdx.x * G + grp;
    const int nchan = g.chan0[g.ngroups];
    const bool live = chan < nchan;
    int gi = 0, l = 0, local = 0;
    if (live) {
        gi = find_group(g, chan);
        l = g.l[gi];
        local = chan - g.chan0[gi];
    }
    const bool even = (l & 1) == 0;
    const int line = live ? g.line0[gi] + (cplx ? 2 * local : local) : 0;
    const R isc1 = (R)sqrt((double)N / 2.0), isc0 = (R)sqrt((double)N);
    // unnormalised DCT-II coefficients X_k (pairs k = 2m, 2m+1); storage pair
    // (idx, idx+1) holds (k, k+1) for odd l and (k+1, k) for even l
    R re[8][2], im[8][2];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int m = lt + u * T;
        re[u][0] = re[u][1] = im[u][0] = im[u][1] = (R)0;
        if (live) {
            const int idx = even ? (N - 2 - 2 * m) : 2 * m;
            const R* li = in + (size_t)line * N;
            ld_real_pair(li + idx, re[u][0], re[u][1]);
            if (cplx) ld_real_pair(li + N + idx, im[u][0], im[u][1]);
        }
    }
    {
        C* dst = s + padi(2 * lt);       // X_{2m}, X_{2m+1} (same padded row), m = lt + u T
        const int st2 = pstride(2 * T);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int m = lt + u * T;
            C X0, X1;
            X0.x = even ? re[u][1] : re[u][0];
            X0.y = even ? im[u][1] : im[u][0];
            X1.x = even ? re[u][0] : re[u][1];
            X1.y = even ? im[u][0] : im[u][1];
            const R s0 = (m == 0) ? isc0 : isc1;
            X0.x *= s0; X0.y *= s0;
            X1.x *= isc1; X1.y *= isc1;
            if (NS > 0) {
                dst[u * st2] = X0;
                dst[u * st2 + 1] = X1;
            } else {
                s[padi(2 * m)] = X0;
                s[padi(2 * m + 1)] = X1;
            }
        }
    }
    __syncthreads();
    // V_k = conj(w_k) (X_k - i X_{N-k}); keep conj(V_k) for the IFFT-by-FFT
    C vk[16];
    const int st1 = pstride(T);
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int k = lt + u * T;
        const C a = NS > 0 ? s[padi(lt) + u * st1] : s[padi(k)];
        C b;
        if (k == 0) { b.x = (R)0; b.y = (R)0; } else b = NS > 0 ? s[padi(N - lt) - u * st1] : s[padi(N - k)];
        C t;   // a - i b
        t.x = a.x + b.y;
        t.y = a.y - b.x;
        const C v = cmulc(t, post[k]);
        vk[u].x = v.x;
        vk[u].y = -v.y;
    }
    __syncthreads();   // every read of X from s is done
    __shared__ C sroot[32];
    fft_from_registers<Q, NS>(s, vk, tw, sroot, N, lt, T);
    if (!live) return;
    const size_t ubase = g.uoff ? (size_t)g.uoff[chan] : (size_t)chan * N;   // caller's element offset
    const R invN = (R)(1.0 / (double)N);
    const C* lo = s + padi(lt);
    const C* hi = s + padi(N - 1 - lt);
    const int st1b = pstride(T);
#pragma unroll
    for (int i = 0; i < 8; ++i) {   // j = lt + i T, N / 2 = 8 T
        const int j = lt + i * T;
        C a = NS > 0 ? lo[i * st1b] : s[padi(j)];             // x_{2j} (conjugated, unscaled)
        C b = NS > 0 ? hi[-i * st1b] : s[padi(N - 1 - j)];    // x_{2j+1}
        a.x *= invN; a.y = -a.y * invN;
        b.x *= invN; b.y = -b.y * invN;
        if (even) { b.x = -b.x; b.y = -b.y; }
        if (cplx) {
            st_pair(reinterpret_cast<C*>(out) + ubase + 2 * j, a, b);
        } else {
            out[ubase + 2 * j] = a.x;
            out[ubase + 2 * j + 1] = b.x;
        }
    }
}

template <typename K>
inline int launch_cfg(K kernel, int N, size_t elem, unsigned& threads, size_t& smem) {
    const int G = lines_per_cta(N);
    threads = (unsigned)(G * (N / 16));
    smem = (size_t)G * (N + N / 16) * elem;
    if (smem > 48 * 1024) return ensure_smem((const void*)kernel, smem);
    return DSBT_OK;
}

inline int nchannels(const GroupTable& g) { return g.chan0[g.ngroups]; }
inline unsigned nblocks(const GroupTable& g, int N) {
    const int G = lines_per_cta(N);
    return (unsigned)((nchannels(g) + G - 1) / G);
}

// Odd part Q of q = N / 256; every N = 256 q with q <= 32 has Q in 1..31.
inline int odd_part(int N) {
    int q = N / 256;
    while (q > 0 && (q & 1) == 0) q >>= 1;
    return q;
}

#define DSBT_DCT_Q_CASES(X) X(1) X(3) X(5) X(7) X(9) X(11) X(13) X(15) X(17) X(19) X(21) X(23) X(25) X(27) X(29) X(31)

template <typename R>
using FwdKernel = void (*)(GroupTable, int, int, const R*, void*, void*, float*, const typename Cx<R>::T*,
                           const typename Cx<R>::T*);
template <typename R>
using InvKernel = void (*)(GroupTable, int, int, const R*, R*, const typename Cx<R>::T*, const typename Cx<R>::T*);

}  // namespace dsbt
