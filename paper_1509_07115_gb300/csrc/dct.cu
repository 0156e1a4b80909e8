// dct.cu -- batched orthonormal sine / cosine transforms F_l and F_l^T.
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
// The FFT is an in-shared-memory Stockham radix-8 (+ one radix-2/4 stage) with
// one CTA per channel; global reads and writes are coalesced along the radial
// index.  Twiddles come from tables built once per plan.
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
    // w8^q o_q, w8 = exp(-i pi/4)
    C t1; t1.x = h * (o1.x + o1.y); t1.y = h * (o1.y - o1.x);
    C t2 = cmi(o2);
    C t3; t3.x = h * (o3.y - o3.x); t3.y = -h * (o3.x + o3.y);
    x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
    x[1] = cadd(e1, t1); x[5] = csub(e1, t1);
    x[2] = cadd(e2, t2); x[6] = csub(e2, t2);
    x[3] = cadd(e3, t3); x[7] = csub(e3, t3);
}

// One Stockham stage of radix RX on the shared buffer s (in place with a
// barrier between the register loads and the stores).  The block has exactly
// N/8 threads, so each thread owns 8/RX butterflies.
template <int RX, typename C>
__device__ __forceinline__ void stockham_stage(C* s, const C* __restrict__ tw, int N, int Ls) {
    constexpr int PER = 8 / RX;
    const int nb = N / RX;
    C x[PER][RX];
    #pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = threadIdx.x + u * blockDim.x;
        const int k = j % Ls;
        const int tstep = (N / (Ls * RX)) * k;
        #pragma unroll
        for (int r = 0; r < RX; ++r) {
            C v = s[j + r * nb];
            if (r > 0 && k > 0) v = cmul(v, tw[r * tstep]);
            x[u][r] = v;
        }
        if (RX == 8) dft8(x[u]);
        else if (RX == 4) dft4(x[u][0], x[u][1], x[u][2], x[u][3]);
        else dft2(x[u][0], x[u][1]);
    }
    __syncthreads();
    #pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int j = threadIdx.x + u * blockDim.x;
        const int k = j % Ls;
        const int base = (j - k) * RX + k;
        #pragma unroll
        for (int q = 0; q < RX; ++q) s[base + q * Ls] = x[u][q];
    }
    __syncthreads();
}

// Forward FFT of length N (power of two, 256..8192) in shared memory.
template <typename C>
__device__ void fft_smem(C* s, const C* __restrict__ tw, int N) {
    int Ls = 1;
    int rem = N;
    while (rem >= 8) {
        stockham_stage<8>(s, tw, N, Ls);
        Ls *= 8;
        rem /= 8;
    }
    if (rem == 4) stockham_stage<4>(s, tw, N, Ls);
    else if (rem == 2) stockham_stage<2>(s, tw, N, Ls);
}

__device__ __forceinline__ int find_group(const GroupTable& g, int chan) {
    int lo = 0, hi = g.ngroups - 1;
    while (lo < hi) {   // last group with chan0 <= chan
        const int mid = (lo + hi + 1) >> 1;
        if (g.chan0[mid] <= chan) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Forward transform.  Output: planar lines.  SPLIT: write TF32 hi/lo pair.
template <typename R, bool SPLIT>
__global__ void k_dct_fwd(GroupTable g, int N, int cplx, const R* __restrict__ in,
                          R* __restrict__ out0, R* __restrict__ out1,
                          const typename Cx<R>::T* __restrict__ tw,
                          const typename Cx<R>::T* __restrict__ post) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int chan = blockIdx.x;
    const int gi = find_group(g, chan);
    const int l = g.l[gi];
    const bool even = (l & 1) == 0;
    const int local = chan - g.chan0[gi];
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        C x;
        if (cplx) x = reinterpret_cast<const C*>(in)[(size_t)chan * N + t];
        else { x.x = in[(size_t)chan * N + t]; x.y = (R)0; }
        if (even && (t & 1)) { x.x = -x.x; x.y = -x.y; }
        const int pos = (t & 1) ? (N - 1 - (t >> 1)) : (t >> 1);
        s[pos] = x;
    }
    __syncthreads();
    fft_smem(s, tw, N);
    const R sc1 = (R)sqrt(2.0 / (double)N), sc0 = (R)sqrt(1.0 / (double)N);
    const int line = g.line0[gi] + (cplx ? 2 * local : local);
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const C a = s[k], b = s[(N - k) & (N - 1)];
        const C w = post[k];
        // X = 1/2 (w a + conj(w) b)
        C X;
        X.x = (R)0.5 * ((w.x * a.x - w.y * a.y) + (w.x * b.x + w.y * b.y));
        X.y = (R)0.5 * ((w.x * a.y + w.y * a.x) + (w.x * b.y - w.y * b.x));
        const R sc = (k == 0) ? sc0 : sc1;
        X.x *= sc;
        X.y *= sc;
        const int idx = even ? (N - 1 - k) : k;
        if (SPLIT) {
            const float hr = round_tf32((float)X.x), hi_ = round_tf32((float)X.y);
            out0[(size_t)line * N + idx] = hr;
            out1[(size_t)line * N + idx] = round_tf32((float)X.x - hr);
            if (cplx) {
                out0[(size_t)(line + 1) * N + idx] = hi_;
                out1[(size_t)(line + 1) * N + idx] = round_tf32((float)X.y - hi_);
            }
        } else {
            out0[(size_t)line * N + idx] = X.x;
            if (cplx) out0[(size_t)(line + 1) * N + idx] = X.y;
        }
    }
}

// Inverse transform F_l^T: planar lines -> caller layout.
template <typename R>
__global__ void k_dct_inv(GroupTable g, int N, int cplx, const R* __restrict__ in,
                          R* __restrict__ out, const typename Cx<R>::T* __restrict__ tw,
                          const typename Cx<R>::T* __restrict__ post) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int chan = blockIdx.x;
    const int gi = find_group(g, chan);
    const int l = g.l[gi];
    const bool even = (l & 1) == 0;
    const int local = chan - g.chan0[gi];
    const int line = g.line0[gi] + (cplx ? 2 * local : local);
    const R isc1 = (R)sqrt((double)N / 2.0), isc0 = (R)sqrt((double)N);
    // unnormalised DCT-II coefficients X_k
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        const int idx = even ? (N - 1 - k) : k;
        C X;
        X.x = in[(size_t)line * N + idx];
        X.y = cplx ? in[(size_t)(line + 1) * N + idx] : (R)0;
        const R sc = (k == 0) ? isc0 : isc1;
        X.x *= sc;
        X.y *= sc;
        s[k] = X;
    }
    __syncthreads();
    // V_k = conj(w_k) (X_k - i X_{N-k}); store conj(V_k) for the IFFT-by-FFT
    C vk[8];
    int cnt = 0;
    for (int k = threadIdx.x; k < N; k += blockDim.x, ++cnt) {
        const C a = s[k];
        C b;
        if (k == 0) { b.x = (R)0; b.y = (R)0; } else b = s[N - k];
        C t;   // a - i b
        t.x = a.x + b.y;
        t.y = a.y - b.x;
        const C v = cmulc(t, post[k]);
        vk[cnt].x = v.x;
        vk[cnt].y = -v.y;
    }
    __syncthreads();
    cnt = 0;
    for (int k = threadIdx.x; k < N; k += blockDim.x, ++cnt) s[k] = vk[cnt];
    __syncthreads();
    fft_smem(s, tw, N);
    const R invN = (R)(1.0 / (double)N);
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        const int pos = (t & 1) ? (N - 1 - (t >> 1)) : (t >> 1);
        C v = s[pos];
        v.x *= invN;
        v.y = -v.y * invN;
        if (even && (t & 1)) { v.x = -v.x; v.y = -v.y; }
        if (cplx) reinterpret_cast<C*>(out)[(size_t)chan * N + t] = v;
        else out[(size_t)chan * N + t] = v.x;
    }
}

template <typename K>
static int launch_cfg(K kernel, int N, size_t elem, unsigned& threads, size_t& smem) {
    threads = (unsigned)(N / 8);   // N >= 256: one radix-8 butterfly per thread
    smem = (size_t)N * elem;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) {
            set_error("dct: cannot opt in %zu bytes of shared memory: %s", smem, cudaGetErrorString(e));
            return DSBT_ERR_CUDA;
        }
    }
    return DSBT_OK;
}

static int nchannels(const GroupTable& g) { return g.chan0[g.ngroups]; }

int dct_forward_f64(const dsbt_plan* p, const GroupTable& g, bool cplx, const double* in,
                    double* out, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    int rc = launch_cfg(k_dct_fwd<double, false>, p->N, sizeof(double2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctFwd, st);
    k_dct_fwd<double, false><<<nchannels(g), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out, nullptr,
                                                           p->tw64, p->post64);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int dct_forward_f32(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in,
                    float* out_hi, float* out_lo, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    int rc = launch_cfg(k_dct_fwd<float, true>, p->N, sizeof(float2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctFwd, st);
    k_dct_fwd<float, true><<<nchannels(g), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out_hi, out_lo,
                                                         p->tw32, p->post32);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int dct_inverse_f64(const dsbt_plan* p, const GroupTable& g, bool cplx, const double* in,
                    double* out, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    int rc = launch_cfg(k_dct_inv<double>, p->N, sizeof(double2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctInv, st);
    k_dct_inv<double><<<nchannels(g), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out, p->tw64, p->post64);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int dct_inverse_f32(const dsbt_plan* p, const GroupTable& g, bool cplx, const float* in,
                    float* out, cudaStream_t st) {
    if (nchannels(g) == 0) return DSBT_OK;
    unsigned th; size_t sm;
    int rc = launch_cfg(k_dct_inv<float>, p->N, sizeof(float2), th, sm);
    if (rc) return rc;
    ProfScope ps(kKDctInv, st);
    k_dct_inv<float><<<nchannels(g), th, sm, st>>>(g, p->N, cplx ? 1 : 0, in, out, p->tw32, p->post32);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

}  // namespace dsbt
