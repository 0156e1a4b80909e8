// tdse3d.cu -- the full DSBT-DVR split-operator step (Sec. 4.1): all m at once,
// angular transform Y = P Phi over a (theta, phi) grid, length gauge with a
// field of any direction.
//
// Channels (l, m): m = -M .. M and, for each m, l = |m| .. |m| + L - 1 (the
// per-m range of the fixed-m propagator, so every P^m below is square),
// stored l-major as the DSBT's grouped calls want them (channel c -> line c).
// Angular grid: the L-point Gauss-Legendre nodes eta_j = cos(theta_j) and
// NM = 2M + 1 uniform angles phi_q = 2 pi q / NM.  The transform of Sec. 4.1
// in two factors:
//     G_m(eta_j)      = sum_l P^m[l - |m|][j] psi_lm          (P^m: Pbar_l^|m| sqrt(w_j),
//                                                               orthonormalised on the rule)
//     g(eta_j, phi_q) = sum_m Phi[m][q] G_m(eta_j),   Phi[m][q] = exp(i m phi_q) / sqrt(NM)
// Both factors are orthogonal / unitary, so Y is unitary on the channel space.
// One step of length tau (vector potential 0, the kinetic half steps merged):
//     psi <- Q Kin Q psi,   Q = Y^H diag exp(-i [V(r) + r F.n(theta, phi)] tau/2) Y,
//     Kin = the grouped DSBT kinetic step (each channel with its own l),
// with n = (sin theta cos phi, sin theta sin phi, cos theta) and F the field
// sample of the step (three components).  A field along z couples no m, and the
// step then equals the fixed-m propagator's for every m.
//
// Adjoint (the gradient of O = sum_{r_i > r_cut} |psi_S|^2 over the field
// samples): with a_s = Q_s psi_s, lambda_S = Pi psi_S (Pi the mask r_i > r_cut),
// nu = Kin^H Q_s^H lambda_{s+1} and lambda_s = Q_s^H nu, the derivative of
// Q_s by the component F_c is Y^H diag(-i r n_c tau/2) D Y, which gives
//     dO/dF_{s,c} += tau Im <Y lambda_{s+1}, r n_c Y psi_{s+1}> + tau Im <Y nu, r n_c Y a_s>
// (the same form as the m = 0 adjoint with eta replaced by n_c), accumulated
// inside the adjoint angular kernel.
#include <math.h>

#include <algorithm>
#include <new>
#include <vector>

#include "plan.cuh"

namespace dsbt {
int kinetic_grouped_with_scratch(const dsbt_plan* p, const int* counts, int dtype, double tau,
                                 const void* in, void* out, void* scratch, size_t scratch_bytes,
                                 cudaStream_t st);
}

struct dsbt_tdse3d {
    const dsbt_plan* plan;
    int L, M, NM, N, nchan;
    double tau;
    double* P;        // [NM][L][L]: P^m (row i = l - |m|, column j), m = mi - M
    int* map;         // [NM][L]: channel of (l = |m| + i, m)
    int* lch;         // [nchan]: l of each channel
    double* V;        // [N]
    double* rr;       // [N]
    double* eta;      // [L]
    std::vector<int> counts;            // channels per l, l = 0 .. plan l_max
    std::vector<int> chan_l, chan_m;    // per channel
};

namespace dsbt {
namespace {

constexpr int TI3 = 4;   // radial points per block of the angular kernel

// y = Q x on TI3 radial points per block (x and y may alias): to the
// (theta, phi) grid, the phase exp(-i [V + r F.n] ht), back.  Shared memory:
// the channel values, G[m][j] and the grid values, each [.][TI3].  With aux
// != nullptr (adjoint steps), also adds gscale * Im( sum conj(Y x) r n_c Y aux )
// over the grid into gacc[c], c = x, y, z (ga: the grid values of aux).
__global__ void __launch_bounds__(256) k_tdse3d_potential(const double2* x, double2* y, const double* __restrict__ P,
                                                          const int* __restrict__ map, const double* __restrict__ V,
                                                          const double* __restrict__ rr,
                                                          const double* __restrict__ eta, int L, int M, int N,
                                                          int nchan, const double* __restrict__ F, int fidx,
                                                          double ht, const double2* __restrict__ aux, double gscale,
                                                          double* gacc) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int NM = 2 * M + 1;
    double2* xs = reinterpret_cast<double2*>(sm);   // [nchan][TI3]
    double2* G = xs + (size_t)nchan * TI3;          // [NM][L][TI3]
    double2* g = G + (size_t)NM * L * TI3;          // [L][NM][TI3]
    double2* ph = g + (size_t)NM * L * TI3;         // [NM][NM]: Phi[m][q]
    double2* ga = ph + (size_t)NM * NM;             // [L][NM][TI3]: grid values of aux (adjoint only)
    __shared__ double red[3][8];
    const int i0 = blockIdx.x * TI3, tid = threadIdx.x;
    const double inv = rsqrt((double)NM);
    for (int k = tid; k < NM * NM; k += blockDim.x) {
        const int mi = k / NM, q = k % NM;
        double sn, cs;
        sincospi(2.0 * (double)((mi - M) * q) / NM, &sn, &cs);
        ph[k] = make_double2(cs * inv, sn * inv);
    }
    if (aux) {   // Y aux -> ga, through the same buffers
        for (int k = tid; k < nchan * TI3; k += blockDim.x) {
            const int c = k / TI3, t = k % TI3, i = i0 + t;
            xs[k] = (i < N) ? aux[(size_t)c * N + i] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        for (int k = tid; k < NM * L * TI3; k += blockDim.x) {
            const int mi = k / (L * TI3), j = (k / TI3) % L, t = k % TI3;
            const double* Pm = P + (size_t)mi * L * L;
            double2 s = make_double2(0.0, 0.0);
            for (int ii = 0; ii < L; ++ii) {
                const double p = Pm[ii * L + j];
                const double2 v = xs[map[mi * L + ii] * TI3 + t];
                s.x = fma(p, v.x, s.x);
                s.y = fma(p, v.y, s.y);
            }
            G[k] = s;
        }
        __syncthreads();
        for (int k = tid; k < L * NM * TI3; k += blockDim.x) {
            const int j = k / (NM * TI3), q = (k / TI3) % NM, t = k % TI3;
            double2 s = make_double2(0.0, 0.0);
            for (int mi = 0; mi < NM; ++mi) {
                const double2 a = ph[mi * NM + q], v = G[(mi * L + j) * TI3 + t];
                s.x = fma(a.x, v.x, fma(-a.y, v.y, s.x));
                s.y = fma(a.x, v.y, fma(a.y, v.x, s.y));
            }
            ga[k] = s;
        }
        __syncthreads();
    }
    for (int k = tid; k < nchan * TI3; k += blockDim.x) {
        const int c = k / TI3, t = k % TI3, i = i0 + t;
        xs[k] = (i < N) ? x[(size_t)c * N + i] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int k = tid; k < NM * L * TI3; k += blockDim.x) {   // G_m(eta_j) = sum_l P^m x_lm
        const int mi = k / (L * TI3), j = (k / TI3) % L, t = k % TI3;
        const double* Pm = P + (size_t)mi * L * L;
        double2 s = make_double2(0.0, 0.0);
        for (int ii = 0; ii < L; ++ii) {
            const double p = Pm[ii * L + j];
            const double2 v = xs[map[mi * L + ii] * TI3 + t];
            s.x = fma(p, v.x, s.x);
            s.y = fma(p, v.y, s.y);
        }
        G[k] = s;
    }
    __syncthreads();
    const double Fx = F ? F[3 * fidx] : 0.0, Fy = F ? F[3 * fidx + 1] : 0.0, Fz = F ? F[3 * fidx + 2] : 0.0;
    double gx = 0.0, gy = 0.0, gz = 0.0;
    for (int k = tid; k < L * NM * TI3; k += blockDim.x) {   // grid values times the phase
        const int j = k / (NM * TI3), q = (k / TI3) % NM, t = k % TI3, i = i0 + t;
        double2 s = make_double2(0.0, 0.0);
        for (int mi = 0; mi < NM; ++mi) {
            const double2 a = ph[mi * NM + q], v = G[(mi * L + j) * TI3 + t];
            s.x = fma(a.x, v.x, fma(-a.y, v.y, s.x));
            s.y = fma(a.x, v.y, fma(a.y, v.x, s.y));
        }
        if (i < N) {
            const double ct = eta[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double sp, cp;
            sincospi(2.0 * (double)q / NM, &sp, &cp);
            if (aux) {   // Im(conj(Y x) Y aux) r n_c
                const double2 va = ga[k];
                const double im = rr[i] * (s.x * va.y - s.y * va.x);
                gx += im * st * cp;
                gy += im * st * sp;
                gz += im * ct;
            }
            const double u = V[i] + rr[i] * (Fx * st * cp + Fy * st * sp + Fz * ct);
            double sn, cs;
            sincos(-u * ht, &sn, &cs);
            s = make_double2(s.x * cs - s.y * sn, s.x * sn + s.y * cs);
        }
        g[k] = s;
    }
    if (aux) {   // block sums of the three components, one atomic each
        for (int o = 16; o > 0; o >>= 1) {
            gx += __shfl_xor_sync(0xffffffffu, gx, o);
            gy += __shfl_xor_sync(0xffffffffu, gy, o);
            gz += __shfl_xor_sync(0xffffffffu, gz, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = gx;
            red[1][tid >> 5] = gy;
            red[2][tid >> 5] = gz;
        }
    }
    __syncthreads();
    if (aux && tid < 3) {
        double tsum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += red[tid][w];
        atomicAdd(gacc + tid, gscale * tsum);
    }
    for (int k = tid; k < NM * L * TI3; k += blockDim.x) {   // back over phi: sum_q conj(Phi[m][q]) g
        const int mi = k / (L * TI3), j = (k / TI3) % L, t = k % TI3;
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < NM; ++q) {
            const double2 a = ph[mi * NM + q], v = g[(j * NM + q) * TI3 + t];
            s.x = fma(a.x, v.x, fma(a.y, v.y, s.x));
            s.y = fma(a.x, v.y, fma(-a.y, v.x, s.y));
        }
        G[k] = s;
    }
    __syncthreads();
    for (int k = tid; k < NM * L * TI3; k += blockDim.x) {   // back over theta: psi_lm = sum_j P^m G_m
        const int mi = k / (L * TI3), ii = (k / TI3) % L, t = k % TI3, i = i0 + t;
        const double* Pm = P + (size_t)mi * L * L + (size_t)ii * L;
        double2 s = make_double2(0.0, 0.0);
        for (int j = 0; j < L; ++j) {
            const double p = Pm[j];
            const double2 v = G[(mi * L + j) * TI3 + t];
            s.x = fma(p, v.x, s.x);
            s.y = fma(p, v.y, s.y);
        }
        if (i < N) y[(size_t)map[mi * L + ii] * N + i] = s;
    }
}

// The momentum-space middle of the velocity-gauge step (Eq. (81)) with all m,
// in place on the DSBT coefficients c[ch][s] at TI3 momentum slots
// n = 1..N per block (k~_n = n dk; storage s = n - 1 for even l, s = n for odd
// l with n = N at s = 0): the half kinetic phase exp(-i k^2 tau/4) with the
// plan's momentum of (l, s); phi = Ytilde^H c with the factors (-i)^l s_l = 1
// (even l) or i (odd l) of the modified harmonics (s_l: this library's
// sine/cosine signs); phi *= exp(i k~_n (A . n) tau) on the (theta, phi) grid;
// c = Ytilde phi with i^l s_l = 1 or -i; the half kinetic phase again.
__global__ void __launch_bounds__(256) k_tdse3d_velocity(double2* c, const double* __restrict__ P,
                                                         const int* __restrict__ map, const int* __restrict__ lch,
                                                         const double* __restrict__ eta,
                                                         const double* __restrict__ knl, double dk, int L, int M,
                                                         int N, int nchan, const double* __restrict__ A, int aidx,
                                                         double tau) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int NM = 2 * M + 1;
    double2* xs = reinterpret_cast<double2*>(sm);   // [nchan][TI3]
    double2* G = xs + (size_t)nchan * TI3;          // [NM][L][TI3]
    double2* g = G + (size_t)NM * L * TI3;          // [L][NM][TI3]
    double2* ph = g + (size_t)NM * L * TI3;         // [NM][NM]
    const int n0 = 1 + blockIdx.x * TI3, tid = threadIdx.x;
    const double inv = rsqrt((double)NM);
    for (int k = tid; k < NM * NM; k += blockDim.x) {
        const int mi = k / NM, q = k % NM;
        double sn, cs;
        sincospi(2.0 * (double)((mi - M) * q) / NM, &sn, &cs);
        ph[k] = make_double2(cs * inv, sn * inv);
    }
    for (int k = tid; k < nchan * TI3; k += blockDim.x) {   // gather, half kinetic phase, (-i)^l s_l
        const int ch = k / TI3, t = k % TI3, n = n0 + t, l = lch[ch];
        double2 v = make_double2(0.0, 0.0);
        if (n <= N) {
            const int sidx = (l & 1) ? (n % N) : n - 1;
            const double km = knl ? knl[(size_t)l * N + sidx] : k_index(l, sidx, N) * dk;
            double sn, cs;
            sincos(-0.25 * km * km * tau, &sn, &cs);
            const double2 a = c[(size_t)ch * N + sidx];
            v = make_double2(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
            if (l & 1) v = make_double2(-v.y, v.x);   // times i
        }
        xs[k] = v;
    }
    __syncthreads();
    for (int k = tid; k < NM * L * TI3; k += blockDim.x) {
        const int mi = k / (L * TI3), j = (k / TI3) % L, t = k % TI3;
        const double* Pm = P + (size_t)mi * L * L;
        double2 s = make_double2(0.0, 0.0);
        for (int ii = 0; ii < L; ++ii) {
            const double p = Pm[ii * L + j];
            const double2 v = xs[map[mi * L + ii] * TI3 + t];
            s.x = fma(p, v.x, s.x);
            s.y = fma(p, v.y, s.y);
        }
        G[k] = s;
    }
    __syncthreads();
    const double Ax = A ? A[3 * aidx] : 0.0, Ay = A ? A[3 * aidx + 1] : 0.0, Az = A ? A[3 * aidx + 2] : 0.0;
    for (int k = tid; k < L * NM * TI3; k += blockDim.x) {   // A . p phase on the momentum grid
        const int j = k / (NM * TI3), q = (k / TI3) % NM, t = k % TI3, n = n0 + t;
        double2 s = make_double2(0.0, 0.0);
        for (int mi = 0; mi < NM; ++mi) {
            const double2 a = ph[mi * NM + q], v = G[(mi * L + j) * TI3 + t];
            s.x = fma(a.x, v.x, fma(-a.y, v.y, s.x));
            s.y = fma(a.x, v.y, fma(a.y, v.x, s.y));
        }
        if (n <= N) {
            const double ct = eta[j], st = sqrt(fmax(0.0, 1.0 - ct * ct));
            double sp, cp;
            sincospi(2.0 * (double)q / NM, &sp, &cp);
            const double an = Ax * st * cp + Ay * st * sp + Az * ct;
            double sn, cs;
            sincos(an * (n * dk) * tau, &sn, &cs);
            s = make_double2(s.x * cs - s.y * sn, s.x * sn + s.y * cs);
        }
        g[k] = s;
    }
    __syncthreads();
    for (int k = tid; k < NM * L * TI3; k += blockDim.x) {
        const int mi = k / (L * TI3), j = (k / TI3) % L, t = k % TI3;
        double2 s = make_double2(0.0, 0.0);
        for (int q = 0; q < NM; ++q) {
            const double2 a = ph[mi * NM + q], v = g[(j * NM + q) * TI3 + t];
            s.x = fma(a.x, v.x, fma(a.y, v.y, s.x));
            s.y = fma(a.x, v.y, fma(-a.y, v.x, s.y));
        }
        G[k] = s;
    }
    __syncthreads();
    for (int k = tid; k < NM * L * TI3; k += blockDim.x) {   // back to (l, m), i^l s_l, half phase, scatter
        const int mi = k / (L * TI3), ii = (k / TI3) % L, t = k % TI3, n = n0 + t;
        if (n > N) continue;
        const double* Pm = P + (size_t)mi * L * L + (size_t)ii * L;
        double2 s = make_double2(0.0, 0.0);
        for (int j = 0; j < L; ++j) {
            const double p = Pm[j];
            const double2 v = G[(mi * L + j) * TI3 + t];
            s.x = fma(p, v.x, s.x);
            s.y = fma(p, v.y, s.y);
        }
        const int ch = map[mi * L + ii], l = lch[ch];
        if (l & 1) s = make_double2(s.y, -s.x);   // times -i
        const int sidx = (l & 1) ? (n % N) : n - 1;
        const double km = knl ? knl[(size_t)l * N + sidx] : k_index(l, sidx, N) * dk;
        double sn, cs;
        sincos(-0.25 * km * km * tau, &sn, &cs);
        c[(size_t)ch * N + sidx] = make_double2(s.x * cs - s.y * sn, s.x * sn + s.y * cs);
    }
}

size_t smem3d(const dsbt_tdse3d* t) {
    return ((size_t)t->nchan * TI3 + 2 * (size_t)t->NM * t->L * TI3 + (size_t)t->NM * t->NM) * sizeof(double2);
}

// Shared memory of the adjoint angular kernel: plus the grid values of aux.
size_t smem3d_adj(const dsbt_tdse3d* t) { return smem3d(t) + (size_t)t->NM * t->L * TI3 * sizeof(double2); }

int potential3d(const dsbt_tdse3d* t, const double2* x, double2* y, const double* F, int fidx, double ht,
                cudaStream_t st, const double2* aux = nullptr, double gscale = 0.0, double* gacc = nullptr) {
    const size_t smem = aux ? smem3d_adj(t) : smem3d(t);
    if (smem > 48 * 1024)
        if (int rc0 = ensure_smem((const void*)k_tdse3d_potential, smem)) return rc0;
    ProfScope ps(kKTdsePot, st);
    k_tdse3d_potential<<<(t->N + TI3 - 1) / TI3, 256, smem, st>>>(x, y, t->P, t->map, t->V, t->rr, t->eta, t->L,
                                                                  t->M, t->N, t->nchan, F, fidx, ht, aux, gscale,
                                                                  gacc);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

// *out += sum over r_i > r_cut of |x|^2 (all channels); with mask != nullptr
// also mask = x on r_i > r_cut and 0 elsewhere (the adjoint start Pi psi_S).
__global__ void k_tdse3d_observable(const double2* __restrict__ x, double2* __restrict__ mask,
                                    const double* __restrict__ rr, int N, long long total, double r_cut,
                                    double* out) {
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        const bool in = rr[k % N] > r_cut;
        const double2 v = x[k];
        if (in) acc += v.x * v.x + v.y * v.y;
        if (mask) mask[k] = in ? v : make_double2(0.0, 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ double red[8];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tsum += red[w];
        atomicAdd(out, tsum);
    }
}

int observable3d(const dsbt_tdse3d* t, const double2* x, double2* mask, double r_cut, double* out, cudaStream_t st) {
    const long long total = (long long)t->nchan * t->N;
    ProfScope ps(kKTdseReduce, st);
    k_tdse3d_observable<<<256, 256, 0, st>>>(x, mask, t->rr, t->N, total, r_cut, out);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int velocity3d(const dsbt_tdse3d* t, double2* c, const double* A, int aidx, cudaStream_t st) {
    const size_t smem = smem3d(t);
    if (smem > 48 * 1024)
        if (int rc0 = ensure_smem((const void*)k_tdse3d_velocity, smem)) return rc0;
    ProfScope ps(kKTdseAng, st);
    k_tdse3d_velocity<<<(t->N + TI3 - 1) / TI3, 256, smem, st>>>(c, t->P, t->map, t->lch, t->eta, t->plan->knl,
                                                                 t->plan->dk, t->L, t->M, t->N, t->nchan, A, aidx,
                                                                 t->tau);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace dsbt

using namespace dsbt;

extern "C" int dsbt_tdse3d_create(const dsbt_plan* plan, int L, int M, double tau, dsbt_tdse3d** out) {
    DSBT_CHECK_ARG(out != nullptr && plan != nullptr, "dsbt_tdse3d_create: NULL argument");
    *out = nullptr;
    DSBT_CHECK_ARG(plan->T64 != nullptr, "dsbt_tdse3d_create: the plan needs DSBT_PLAN_FP64");
    DSBT_CHECK_ARG(L >= 1 && L <= 32, "dsbt_tdse3d_create: L=%d not in 1..32", L);
    DSBT_CHECK_ARG(M >= 0 && M <= 12, "dsbt_tdse3d_create: M=%d not in 0..12", M);
    DSBT_CHECK_ARG(M + L - 1 <= plan->l_max, "dsbt_tdse3d_create: channels up to l=%d, plan l_max=%d", M + L - 1,
                   plan->l_max);
    DSBT_CHECK_ARG(isfinite(tau), "dsbt_tdse3d_create: tau must be finite");
    dsbt_tdse3d* t = new (std::nothrow) dsbt_tdse3d();
    if (!t) return DSBT_ERR_NOMEM;
    t->plan = plan;
    t->L = L;
    t->M = M;
    t->NM = 2 * M + 1;
    t->N = plan->N;
    t->tau = tau;
    // channels, l-major
    std::vector<int> map((size_t)t->NM * L, -1);
    t->counts.assign(plan->l_max + 1, 0);
    for (int l = 0; l <= M + L - 1; ++l)
        for (int mi = 0; mi < t->NM; ++mi) {
            const int m = mi - M, am = m < 0 ? -m : m;
            if (l < am || l > am + L - 1) continue;
            map[(size_t)mi * L + (l - am)] = (int)t->chan_l.size();
            t->chan_l.push_back(l);
            t->chan_m.push_back(m);
            ++t->counts[l];
        }
    t->nchan = (int)t->chan_l.size();
    std::vector<double> x, w, Pm, Pall((size_t)t->NM * L * L), rr(t->N);
    tdse_gauss_legendre(L, x, w);
    for (int mi = 0; mi < t->NM; ++mi) {
        const int am = std::abs(mi - M);
        tdse_angular_rows(L, am, x, w, Pm);
        std::copy(Pm.begin(), Pm.end(), Pall.begin() + (size_t)mi * L * L);
    }
    const double dr = plan->r_max / plan->N;
    for (int i = 0; i < t->N; ++i) rr[i] = (i + 0.5) * dr;
    bool ok = cudaMalloc((void**)&t->P, Pall.size() * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&t->map, map.size() * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&t->lch, t->nchan * sizeof(int)) == cudaSuccess &&
              cudaMalloc((void**)&t->V, t->N * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&t->rr, t->N * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&t->eta, L * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemcpy(t->P, Pall.data(), Pall.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->map, map.data(), map.size() * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->lch, t->chan_l.data(), t->nchan * sizeof(int), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(t->V, 0, t->N * sizeof(double)) == cudaSuccess &&
         cudaMemcpy(t->rr, rr.data(), t->N * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->eta, x.data(), L * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(t->P); cudaFree(t->map); cudaFree(t->lch); cudaFree(t->V); cudaFree(t->rr); cudaFree(t->eta);
        delete t;
        set_error("dsbt_tdse3d_create: device allocation or copy failed");
        return DSBT_ERR_NOMEM;
    }
    if (smem3d(t) > 200 * 1024) {
        cudaFree(t->P); cudaFree(t->map); cudaFree(t->lch); cudaFree(t->V); cudaFree(t->rr); cudaFree(t->eta);
        delete t;
        set_error("dsbt_tdse3d_create: L=%d, M=%d need too much shared memory", L, M);
        return DSBT_ERR_INVALID;
    }
    *out = t;
    return DSBT_OK;
}

extern "C" int dsbt_tdse3d_destroy(dsbt_tdse3d* t) {
    if (!t) return DSBT_OK;
    cudaDeviceSynchronize();
    cudaFree(t->P);
    cudaFree(t->map);
    cudaFree(t->lch);
    cudaFree(t->V);
    cudaFree(t->rr);
    cudaFree(t->eta);
    delete t;
    return DSBT_OK;
}

extern "C" int dsbt_tdse3d_channels(const dsbt_tdse3d* t, int* nchan, int* l_of, int* m_of) {
    DSBT_CHECK_ARG(t != nullptr, "dsbt_tdse3d_channels: NULL handle");
    if (nchan) *nchan = t->nchan;
    for (int c = 0; c < t->nchan; ++c) {
        if (l_of) l_of[c] = t->chan_l[c];
        if (m_of) m_of[c] = t->chan_m[c];
    }
    return DSBT_OK;
}

extern "C" int dsbt_tdse3d_set_potential(dsbt_tdse3d* t, const double* V, int n) {
    DSBT_CHECK_ARG(t != nullptr && V != nullptr, "dsbt_tdse3d_set_potential: NULL argument");
    DSBT_CHECK_ARG(n == t->N, "dsbt_tdse3d_set_potential: n=%d, grid has N=%d", n, t->N);
    DSBT_CUDA_TRY(cudaMemcpy(t->V, V, t->N * sizeof(double), cudaMemcpyHostToDevice));
    return DSBT_OK;
}

extern "C" size_t dsbt_tdse3d_workspace_size(const dsbt_tdse3d* t) {
    if (!t) return 0;
    return 2 * a256((size_t)t->nchan * t->N * sizeof(double2)) +
           dsbt_workspace_size(t->plan, t->nchan, DSBT_C128) + 512;
}

extern "C" int dsbt_tdse3d_propagate(const dsbt_tdse3d* t, void* psi, const double* F, int nsteps, int hold,
                                     void* workspace, size_t workspace_bytes, void* stream) {
    DSBT_CHECK_ARG(t != nullptr && psi != nullptr, "dsbt_tdse3d_propagate: NULL argument");
    DSBT_CHECK_ARG(nsteps >= 0 && hold >= 1, "dsbt_tdse3d_propagate: nsteps >= 0 and hold >= 1 required");
    const size_t need = dsbt_tdse3d_workspace_size(t);
    DSBT_CHECK_ARG(workspace != nullptr && workspace_bytes >= need,
                   "dsbt_tdse3d_propagate: workspace too small (need %zu bytes)", need);
    cudaStream_t st = (cudaStream_t)stream;
    unsigned char* base = (unsigned char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    double2* tmp = (double2*)base;
    void* kws = base + 2 * a256((size_t)t->nchan * t->N * sizeof(double2));
    const size_t kws_b = dsbt_workspace_size(t->plan, t->nchan, DSBT_C128);
    double2* x = (double2*)psi;
    for (int s = 0; s < nsteps; ++s) {
        const int fidx = s / hold;
        int rc = potential3d(t, x, tmp, F, fidx, 0.5 * t->tau, st);
        if (!rc) rc = kinetic_grouped_with_scratch(t->plan, t->counts.data(), DSBT_C128, t->tau, tmp, x, kws, kws_b, st);
        if (!rc) rc = potential3d(t, x, x, F, fidx, 0.5 * t->tau, st);
        if (rc) return rc;
    }
    return DSBT_OK;
}

extern "C" int dsbt_tdse3d_propagate_velocity(const dsbt_tdse3d* t, void* psi, const double* F, const double* A,
                                              int nsteps, int hold, void* workspace, size_t workspace_bytes,
                                              void* stream) {
    DSBT_CHECK_ARG(t != nullptr && psi != nullptr, "dsbt_tdse3d_propagate_velocity: NULL argument");
    DSBT_CHECK_ARG(nsteps >= 0 && hold >= 1, "dsbt_tdse3d_propagate_velocity: nsteps >= 0 and hold >= 1 required");
    const size_t need = dsbt_tdse3d_workspace_size(t);
    DSBT_CHECK_ARG(workspace != nullptr && workspace_bytes >= need,
                   "dsbt_tdse3d_propagate_velocity: workspace too small (need %zu bytes)", need);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t sb = a256((size_t)t->nchan * t->N * sizeof(double2));
    unsigned char* base = (unsigned char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    double2* tmp = (double2*)base;
    double2* c = (double2*)(base + sb);
    void* kws = base + 2 * sb;
    const size_t kws_b = dsbt_workspace_size(t->plan, t->nchan, DSBT_C128);
    double2* x = (double2*)psi;
    for (int s = 0; s < nsteps; ++s) {
        const int idx = s / hold;
        int rc = potential3d(t, x, tmp, F, idx, 0.5 * t->tau, st);
        if (!rc) rc = grouped_device_call(0, t->plan, t->counts.data(), DSBT_C128, 0.0, tmp, c, kws, kws_b, st);
        if (!rc) rc = velocity3d(t, c, A, idx, st);
        if (!rc) rc = grouped_device_call(1, t->plan, t->counts.data(), DSBT_C128, 0.0, c, x, kws, kws_b, st);
        if (!rc) rc = potential3d(t, x, x, F, idx, 0.5 * t->tau, st);
        if (rc) return rc;
    }
    return DSBT_OK;
}

namespace dsbt {
namespace {

// Gradient workspace: nsteps / K + 1 checkpoints, a segment of K + 1 states,
// four more states (a, mu, nu, lambda), one DSBT workspace.
size_t grad3d_layout(const dsbt_tdse3d* t, int nsteps, int K, double2** ck, double2** seg, double2** a, double2** mu,
                     double2** nu, double2** lam, void** kws, void* base) {
    const size_t sb = a256((size_t)t->nchan * t->N * sizeof(double2));
    const size_t nck = (size_t)nsteps / K + 1;
    unsigned char* p = (unsigned char*)(((uintptr_t)base + 255) & ~(uintptr_t)255);
    size_t off = 0;
    auto take = [&](size_t b) { unsigned char* q = p + off; off += a256(b); return q; };
    unsigned char* c0 = take(sb * nck);
    unsigned char* s0 = take(sb * (K + 1));
    unsigned char* a0 = take(sb);
    unsigned char* m0 = take(sb);
    unsigned char* n0 = take(sb);
    unsigned char* l0 = take(sb);
    unsigned char* k0 = take(dsbt_workspace_size(t->plan, t->nchan, DSBT_C128));
    if (base) {
        *ck = (double2*)c0; *seg = (double2*)s0; *a = (double2*)a0; *mu = (double2*)m0; *nu = (double2*)n0;
        *lam = (double2*)l0; *kws = k0;
    }
    return off + 256;
}

}  // namespace
}  // namespace dsbt

extern "C" size_t dsbt_tdse3d_gradient_workspace_size(const dsbt_tdse3d* t, int nsteps, int checkpoint_every) {
    if (!t || nsteps < 0 || checkpoint_every < 1) return 0;
    return grad3d_layout(t, nsteps, checkpoint_every, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                         nullptr);
}

extern "C" int dsbt_tdse3d_gradient(const dsbt_tdse3d* t, const void* psi0, const double* F, int nsamples, int nsteps,
                                    int hold, double r_cut, int checkpoint_every, double* O, double* dOdF,
                                    void* workspace, size_t workspace_bytes, void* stream) {
    DSBT_CHECK_ARG(t != nullptr && psi0 != nullptr && F != nullptr && O != nullptr && dOdF != nullptr,
                   "dsbt_tdse3d_gradient: NULL argument");
    const int K = checkpoint_every;
    DSBT_CHECK_ARG(K >= 1 && nsteps >= 0 && hold >= 1, "dsbt_tdse3d_gradient: K >= 1, nsteps >= 0, hold >= 1");
    DSBT_CHECK_ARG(nsamples >= (nsteps + hold - 1) / hold, "dsbt_tdse3d_gradient: nsamples < ceil(nsteps / hold)");
    const size_t need = dsbt_tdse3d_gradient_workspace_size(t, nsteps, K);
    DSBT_CHECK_ARG(workspace != nullptr && workspace_bytes >= need,
                   "dsbt_tdse3d_gradient: workspace too small (need %zu bytes)", need);
    DSBT_CHECK_ARG(smem3d_adj(t) <= 220 * 1024, "dsbt_tdse3d_gradient: L=%d, M=%d need too much shared memory",
                   t->L, t->M);
    cudaStream_t st = (cudaStream_t)stream;
    double2 *ck, *seg, *a, *mu, *nu, *lam;
    void* kws;
    grad3d_layout(t, nsteps, K, &ck, &seg, &a, &mu, &nu, &lam, &kws, workspace);
    const size_t kws_b = dsbt_workspace_size(t->plan, t->nchan, DSBT_C128);
    const size_t sb = (size_t)t->nchan * t->N * sizeof(double2);
    const size_t stride = a256(sb) / sizeof(double2);
    const double tau = t->tau, ht = 0.5 * tau;
    const int* counts = t->counts.data();
    // one step x -> y (Q Kin Q); tmp is clobbered
    auto step = [&](const double2* x, double2* y, double2* tmp, int fidx) {
        int rc = potential3d(t, x, tmp, F, fidx, ht, st);
        if (!rc) rc = kinetic_grouped_with_scratch(t->plan, counts, DSBT_C128, tau, tmp, y, kws, kws_b, st);
        if (!rc) rc = potential3d(t, y, y, F, fidx, ht, st);
        return rc;
    };
    // forward sweep with checkpoints every K steps
    DSBT_CUDA_TRY(cudaMemcpyAsync(ck, psi0, sb, cudaMemcpyDeviceToDevice, st));
    DSBT_CUDA_TRY(cudaMemcpyAsync(lam, psi0, sb, cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < nsteps; ++s) {
        int rc = step(lam, a, mu, s / hold);
        if (rc) return rc;
        std::swap(lam, a);
        if ((s + 1) % K == 0)
            DSBT_CUDA_TRY(cudaMemcpyAsync(ck + (size_t)((s + 1) / K) * stride, lam, sb, cudaMemcpyDeviceToDevice, st));
    }
    // observable and lambda_S = Pi psi_S
    DSBT_CUDA_TRY(cudaMemsetAsync(O, 0, sizeof(double), st));
    int rc = observable3d(t, lam, mu, r_cut, O, st);
    if (rc) return rc;
    std::swap(lam, mu);
    DSBT_CUDA_TRY(cudaMemsetAsync(dOdF, 0, (size_t)3 * nsamples * sizeof(double), st));
    // backward sweep, one checkpoint segment at a time
    const int nseg = (nsteps + K - 1) / K;
    for (int sg = nseg - 1; sg >= 0; --sg) {
        const int s0 = sg * K, s1 = (s0 + K < nsteps) ? s0 + K : nsteps;
        DSBT_CUDA_TRY(cudaMemcpyAsync(seg, ck + (size_t)sg * stride, sb, cudaMemcpyDeviceToDevice, st));
        for (int s = s0; s < s1; ++s) {
            rc = step(seg + (size_t)(s - s0) * stride, seg + (size_t)(s - s0 + 1) * stride, a, s / hold);
            if (rc) return rc;
        }
        for (int s = s1 - 1; s >= s0; --s) {
            const double2* psi_s = seg + (size_t)(s - s0) * stride;
            const double2* psi_s1 = seg + (size_t)(s - s0 + 1) * stride;
            double* g = dOdF + 3 * (size_t)(s / hold);
            // a_s = Q_s psi_s
            rc = potential3d(t, psi_s, a, F, s / hold, ht, st);
            // mu = Q_s^H lambda_{s+1};  dO/dF += tau Im <Y lambda_{s+1}, r n Y psi_{s+1}>
            if (!rc) rc = potential3d(t, lam, mu, F, s / hold, -ht, st, psi_s1, tau, g);
            // nu = Kin^H mu
            if (!rc) rc = kinetic_grouped_with_scratch(t->plan, counts, DSBT_C128, -tau, mu, nu, kws, kws_b, st);
            // lambda_s = Q_s^H nu;  dO/dF += tau Im <Y nu, r n Y a_s>
            if (!rc) rc = potential3d(t, nu, lam, F, s / hold, -ht, st, a, tau, g);
            if (rc) return rc;
        }
    }
    return DSBT_OK;
}
