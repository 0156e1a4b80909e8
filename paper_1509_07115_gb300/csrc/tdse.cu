// tdse.cu -- split-operator TDSE step through the DSBT (m = 0, length gauge)
// and its adjoint.
//
// State: psi[l][i], l = 0..L-1, i = 0..N-1, complex128, in the l representation
// (channel l is the radial function of angular momentum l; the DSBT layout).
// One step of length tau (Sec. 4.1, Eq. (81), vector potential A = 0, so the two
// kinetic half steps merge):
//     psi <- Q_s Kin Q_s psi,
//     Q_s = P diag_j exp(-i [V(r_i) + E_s r_i eta_j] tau/2) P^T       (angular grid)
//     Kin = B^T exp(-i K tau) B,  B = T_l F_l per l,  K = k~_n^2 / 2    (dsbt_kinetic)
// with eta_j, w_j the L-point Gauss-Legendre rule and P[l][j] =
// Pbar_l(eta_j) sqrt(w_j) the orthonormal angular transform of Sec. 4.1
// (associated Legendre functions for m = 0), V(r) = -Z / sqrt(r^2 + a2).
//
// Adjoint: every factor is unitary and B, P are real orthogonal (Eq. (25),
// T^{-1} = T^T), so U_s^H = Q_s^H Kin^H Q_s^H is the same step with tau -> -tau.
// For the observable O = sum_{r_i > r_cut} |psi_S|^2 and lambda_S = Pi psi_S:
//     mu = Q_s^H lambda_{s+1},  nu = Kin^H mu,  lambda_s = Q_s^H nu,
//     dO/dE_s = tau Im( <lambda_{s+1}, R psi_{s+1}> + <nu, R a_s> ),  a_s = Q_s psi_s,
// where R = diag(r_i eta_j) on the angular grid (the field coupling r cos(theta)).
// The inner products are accumulated inside the potential kernel from the
// angular-grid values it already holds.
#include <math.h>

#include <new>
#include <algorithm>
#include <vector>

#include "plan.cuh"

namespace dsbt {

int kinetic_grouped_with_scratch(const dsbt_plan* p, const int* counts, int dtype, double tau,
                                 const void* in, void* out, void* scratch, size_t scratch_bytes,
                                 cudaStream_t st);

}  // namespace dsbt

struct dsbt_tdse {
    const dsbt_plan* plan;
    int L, N;
    int m0;         // |m|: channels are l = m0 .. m0 + L - 1
    double dr, tau, Z, a2;
    double* P;      // [L][L] angular transform
    double* V;      // [N] potential
    double* rr;     // [N] radii
    double* eta;    // [L] nodes
    std::vector<double> eta_h, w_h;
};

namespace dsbt {

namespace {

constexpr int TI = 16;          // radial points per tile of the angular kernel
constexpr int kLMax = 64;

// Gauss-Legendre nodes and weights by Newton's method on P_L (three-term
// recurrence for P_L and its derivative).
void gauss_legendre(int L, std::vector<double>& x, std::vector<double>& w) {
    x.assign(L, 0.0);
    w.assign(L, 0.0);
    for (int j = 0; j < L; ++j) {
        double z = cos(M_PI * (j + 0.75) / (L + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= L; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            double pL = (L == 1) ? z : p1, pLm1 = (L == 1) ? 1.0 : p0;
            if (L == 1) { pL = z; pLm1 = 1.0; }
            dp = L * (z * pL - pLm1) / (z * z - 1.0);
            const double dz = pL / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        // final derivative at the converged node
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= L; ++k) {
            const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = (L == 1) ? 1.0 : L * (z * p1 - p0) / (z * z - 1.0);
        x[j] = z;
        w[j] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// P[l][j] = sqrt((2l+1)/2) P_l(eta_j) sqrt(w_j).
void angular_matrix(int L, const std::vector<double>& x, const std::vector<double>& w,
                    std::vector<double>& P) {
    P.assign((size_t)L * L, 0.0);
    for (int j = 0; j < L; ++j) {
        double p0 = 1.0, p1 = x[j];
        for (int l = 0; l < L; ++l) {
            double pl;
            if (l == 0) pl = 1.0;
            else if (l == 1) pl = x[j];
            else {
                const double p2 = ((2.0 * l - 1.0) * x[j] * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = p2;
                pl = p2;
            }
            P[(size_t)l * L + j] = sqrt((2.0 * l + 1.0) / 2.0) * pl * sqrt(w[j]);
        }
    }
}

// m != 0: rows l = m .. m + L - 1 of the normalised associated Legendre
// functions Pbar_l^m(eta_j) sqrt(w_j) (recurrence in l from Pbar_m^m), then
// orthonormalised on the L-point rule by modified Gram-Schmidt in order of l
// (the L-point rule integrates their products exactly only for m = 0).
void angular_matrix_m(int L, int m, const std::vector<double>& x, const std::vector<double>& w,
                      std::vector<double>& P) {
    P.assign((size_t)L * L, 0.0);
    for (int j = 0; j < L; ++j) {
        const double z = x[j], sq = sqrt(std::max(0.0, 1.0 - z * z));
        // Pbar_m^m = sqrt((2m+1)!! / (2 (2m)!!)) (1 - z^2)^(m/2) (Condon-Shortley sign dropped)
        double pmm = sqrt(0.5);
        for (int k = 1; k <= m; ++k) pmm *= sqrt((2.0 * k + 1.0) / (2.0 * k)) * sq;
        double pa = pmm, pb = (L > 1) ? sqrt(2.0 * m + 3.0) * z * pmm : 0.0;   // Pbar_m^m, Pbar_{m+1}^m
        for (int i = 0; i < L; ++i) {
            const int l = m + i;
            double pl;
            if (i == 0) pl = pa;
            else if (i == 1) pl = pb;
            else {
                const double a = sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                const double b = sqrt(((l - 1.0) * (l - 1.0) - (double)m * m) / (4.0 * (l - 1.0) * (l - 1.0) - 1.0));
                pl = a * (z * pb - b * pa);
                pa = pb;
                pb = pl;
            }
            P[(size_t)i * L + j] = pl * sqrt(w[j]);
        }
    }
    for (int i = 0; i < L; ++i) {   // modified Gram-Schmidt of the rows
        double* ri = P.data() + (size_t)i * L;
        for (int k = 0; k < i; ++k) {
            const double* rk = P.data() + (size_t)k * L;
            double d = 0.0;
            for (int j = 0; j < L; ++j) d += ri[j] * rk[j];
            for (int j = 0; j < L; ++j) ri[j] -= d * rk[j];
        }
        double q = 0.0;
        for (int j = 0; j < L; ++j) q += ri[j] * ri[j];
        const double inv = 1.0 / sqrt(q);
        for (int j = 0; j < L; ++j) ri[j] *= inv;
    }
}

__device__ __forceinline__ double2 cmul2(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// y = P diag(exp(-i [V + E r eta] ht)) P^T x on a tile of TI radial points
// (ht = +tau/2 forward, -tau/2 adjoint).  With aux != nullptr, also adds
// gscale * Im( sum conj(x_eta) r eta aux_eta ) into *gacc.  x and y may alias.
__global__ void __launch_bounds__(256) k_tdse_potential(const double2* __restrict__ x, double2* y,
                                                        const double* __restrict__ P,
                                                        const double* __restrict__ V,
                                                        const double* __restrict__ rr,
                                                        const double* __restrict__ eta, int L, int N,
                                                        const double* __restrict__ E, int eidx, double ht,
                                                        const double2* __restrict__ aux, double gscale,
                                                        double* gacc) {
    extern __shared__ __align__(16) unsigned char sm[];
    double* Ps = reinterpret_cast<double*>(sm);                    // [L][L]
    double2* xs = reinterpret_cast<double2*>(Ps + kLMax * kLMax);  // [L][TI]
    double2* xe = xs + kLMax * TI;                                 // [L][TI]
    double2* as = xe + kLMax * TI;                                 // [L][TI]
    __shared__ double red[2][8];
    const int i0 = blockIdx.x * TI;
    const int tid = threadIdx.x;
    for (int k = tid; k < L * L; k += blockDim.x) Ps[k] = P[k];
    for (int k = tid; k < L * TI; k += blockDim.x) {
        const int l = k / TI, t = k % TI;
        const int i = i0 + t;
        xs[k] = (i < N) ? x[(size_t)l * N + i] : make_double2(0.0, 0.0);
        if (aux) as[k] = (i < N) ? aux[(size_t)l * N + i] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    const double Ev = E ? E[eidx] : 0.0;
    double gim = 0.0;
    for (int k = tid; k < L * TI; k += blockDim.x) {   // to the angular grid
        const int j = k / TI, t = k % TI;
        double2 s = make_double2(0.0, 0.0), sa = make_double2(0.0, 0.0);
        for (int l = 0; l < L; ++l) {
            const double pj = Ps[l * L + j];
            const double2 v = xs[l * TI + t];
            s.x = fma(pj, v.x, s.x);
            s.y = fma(pj, v.y, s.y);
            if (aux) {
                const double2 va = as[l * TI + t];
                sa.x = fma(pj, va.x, sa.x);
                sa.y = fma(pj, va.y, sa.y);
            }
        }
        const int i = i0 + t;
        if (i < N) {
            const double r = rr[i];
            if (aux) gim += r * eta[j] * (s.x * sa.y - s.y * sa.x);   // Im(conj(s) sa) r eta
            double sn, cs;
            sincos(-(V[i] + Ev * r * eta[j]) * ht, &sn, &cs);
            s = cmul2(s, make_double2(cs, sn));
        }
        xe[k] = s;
    }
    __syncthreads();
    for (int k = tid; k < L * TI; k += blockDim.x) {   // back to l
        const int l = k / TI, t = k % TI;
        double2 s = make_double2(0.0, 0.0);
        for (int j = 0; j < L; ++j) {
            const double pl = Ps[l * L + j];
            const double2 v = xe[j * TI + t];
            s.x = fma(pl, v.x, s.x);
            s.y = fma(pl, v.y, s.y);
        }
        const int i = i0 + t;
        if (i < N) y[(size_t)l * N + i] = s;
    }
    if (aux) {
        for (int o = 16; o > 0; o >>= 1) gim += __shfl_xor_sync(0xffffffffu, gim, o);
        if ((tid & 31) == 0) red[0][tid >> 5] = gim;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[0][w];
            atomicAdd(gacc, gscale * t);
        }
    }
}

// The momentum-space middle of the velocity-gauge step (Eq. (81)) on a tile of
// TI momentum slots n = 1..N (k~_n = n dk, Eq. (65)), in place on the DSBT
// coefficients c[l][s] (storage s = n - 1 for even l; s = n for odd l, with
// n = N stored at s = 0):
//   half kinetic phase exp(-i k^2 tau/4)  (k = the plan's momentum of (l, s)),
//   phi = Ytilde^dagger c  (phi_j = sum_l (-i)^l s_l P[l][j] c_l),
//   phi_j *= exp(i A k~_n eta_j tau),
//   c = Ytilde phi  (c_l = i^l s_l sum_j P[l][j] phi_j),  half kinetic phase.
// s_l = (-1)^ceil(l/2) converts this library's sine/cosine sign convention to
// the spherical-wave coefficients of Ytilde, so (-i)^l s_l = 1 (even l) or i
// (odd l).  A is the vector potential sample of this step.
__global__ void __launch_bounds__(256) k_tdse_velocity(double2* c, const double* __restrict__ P,
                                                       const double* __restrict__ eta,
                                                       const double* __restrict__ knl, double dk, int L,
                                                       int N, const double* __restrict__ A, int aidx,
                                                       double tau, int m0) {
    extern __shared__ __align__(16) unsigned char sm[];
    double* Ps = reinterpret_cast<double*>(sm);                    // [L][L]
    double2* xs = reinterpret_cast<double2*>(Ps + kLMax * kLMax);  // [L][TI]
    double2* xe = xs + kLMax * TI;                                 // [L][TI]
    const int n0 = 1 + blockIdx.x * TI;
    const int tid = threadIdx.x;
    for (int k = tid; k < L * L; k += blockDim.x) Ps[k] = P[k];
    for (int k = tid; k < L * TI; k += blockDim.x) {   // gather, half kinetic phase, (-i)^l s_l
        const int ch = k / TI, t = k % TI, l = m0 + ch;   // channel ch holds angular momentum l
        const int n = n0 + t;
        double2 v = make_double2(0.0, 0.0);
        if (n <= N) {
            const int sidx = (l & 1) ? (n % N) : n - 1;
            const double km = knl ? knl[(size_t)l * N + sidx] : k_index(l, sidx, N) * dk;
            double sn, cs;
            sincos(-0.25 * km * km * tau, &sn, &cs);
            v = cmul2(c[(size_t)ch * N + sidx], make_double2(cs, sn));
            if (l & 1) v = make_double2(-v.y, v.x);   // times i
        }
        xs[k] = v;
    }
    __syncthreads();
    const double Av = A ? A[aidx] : 0.0;
    for (int k = tid; k < L * TI; k += blockDim.x) {   // to the angular grid, A . P phase
        const int j = k / TI, t = k % TI;
        double2 s = make_double2(0.0, 0.0);
        for (int l = 0; l < L; ++l) {
            const double pj = Ps[l * L + j];
            const double2 v = xs[l * TI + t];
            s.x = fma(pj, v.x, s.x);
            s.y = fma(pj, v.y, s.y);
        }
        const int n = n0 + t;
        if (n <= N) {
            double sn, cs;
            sincos(Av * (n * dk) * eta[j] * tau, &sn, &cs);
            s = cmul2(s, make_double2(cs, sn));
        }
        xe[k] = s;
    }
    __syncthreads();
    for (int k = tid; k < L * TI; k += blockDim.x) {   // back to l, i^l s_l, half kinetic phase, scatter
        const int ch = k / TI, t = k % TI, l = m0 + ch;
        const int n = n0 + t;
        if (n > N) continue;
        double2 s = make_double2(0.0, 0.0);
        for (int j = 0; j < L; ++j) {
            const double pl = Ps[ch * L + j];
            const double2 v = xe[j * TI + t];
            s.x = fma(pl, v.x, s.x);
            s.y = fma(pl, v.y, s.y);
        }
        if (l & 1) s = make_double2(s.y, -s.x);   // times -i
        const int sidx = (l & 1) ? (n % N) : n - 1;
        const double km = knl ? knl[(size_t)l * N + sidx] : k_index(l, sidx, N) * dk;
        double sn, cs;
        sincos(-0.25 * km * km * tau, &sn, &cs);
        c[(size_t)ch * N + sidx] = cmul2(s, make_double2(cs, sn));
    }
}

// out += sum_{r_i > rc} sum_l |x[l][i]|^2 ; with lam != nullptr also writes
// lam = x on r_i > rc and 0 elsewhere (the projector Pi).
__global__ void k_tdse_observable(const double2* __restrict__ x, double2* __restrict__ lam,
                                  const double* __restrict__ rr, int L, int N, double rc,
                                  double* __restrict__ out) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (k < (long long)L * N) {
        const int i = (int)(k % N);
        const double2 a = x[k];
        const bool in = rr[i] > rc;
        if (in) v = a.x * a.x + a.y * a.y;
        if (lam) lam[k] = in ? a : make_double2(0.0, 0.0);
    }
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out, v);
}

size_t state_bytes(const dsbt_tdse* t) { return (size_t)t->L * t->N * sizeof(double2); }

}  // namespace

void tdse_gauss_legendre(int L, std::vector<double>& x, std::vector<double>& w) { gauss_legendre(L, x, w); }
void tdse_angular_rows(int L, int m, const std::vector<double>& x, const std::vector<double>& w,
                       std::vector<double>& P) {
    angular_matrix_m(L, m, x, w, P);
}

namespace {

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int potential(const dsbt_tdse* t, const double2* x, double2* y, const double* E, int eidx, double ht,
              const double2* aux, double gscale, double* gacc, cudaStream_t st) {
    const size_t smem = (size_t)kLMax * kLMax * sizeof(double) + 3 * (size_t)kLMax * TI * sizeof(double2);
    if (int rc0 = ensure_smem((const void*)k_tdse_potential, smem)) return rc0;
    ProfScope ps(kKTdsePot, st);
    k_tdse_potential<<<(t->N + TI - 1) / TI, 256, smem, st>>>(x, y, t->P, t->V, t->rr, t->eta, t->L, t->N, E,
                                                              eidx, ht, aux, gscale, gacc);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

int observable(const dsbt_tdse* t, const double2* x, double2* lam, double rc, double* out, cudaStream_t st) {
    const long long n = (long long)t->L * t->N;
    ProfScope ps(kKTdseReduce, st);
    k_tdse_observable<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, lam, t->rr, t->L, t->N, rc, out);
    DSBT_CUDA_TRY(cudaGetLastError());
    return DSBT_OK;
}

// One forward step psi_in -> psi_out (tmp: one state of scratch).
int step(const dsbt_tdse* t, const double2* in, double2* out, double2* tmp, const double* E, int eidx,
         double tau, const int* counts, void* kws, size_t kws_b, cudaStream_t st) {
    int rc = potential(t, in, tmp, E, eidx, 0.5 * tau, nullptr, 0.0, nullptr, st);
    if (!rc) rc = kinetic_grouped_with_scratch(t->plan, counts, DSBT_C128, tau, tmp, out, kws, kws_b, st);
    if (!rc) rc = potential(t, out, out, E, eidx, 0.5 * tau, nullptr, 0.0, nullptr, st);
    return rc;
}

// One velocity-gauge step (Eq. (81)): potential half step (U = V + E r eta),
// forward DSBT, momentum-space middle (k_tdse_velocity), inverse DSBT,
// potential half step.  c: one state of scratch for the coefficients.
int step_velocity(const dsbt_tdse* t, const double2* in, double2* out, double2* tmp, double2* c,
                  const double* E, const double* A, int idx, double tau, const int* counts, void* kws,
                  size_t kws_b, cudaStream_t st) {
    int rc = potential(t, in, tmp, E, idx, 0.5 * tau, nullptr, 0.0, nullptr, st);
    if (!rc) rc = grouped_device_call(0, t->plan, counts, DSBT_C128, 0.0, tmp, c, kws, kws_b, st);
    if (rc) return rc;
    {
        const size_t smem = (size_t)kLMax * kLMax * sizeof(double) + 2 * (size_t)kLMax * TI * sizeof(double2);
        if (int rc0 = ensure_smem((const void*)k_tdse_velocity, smem)) return rc0;
        ProfScope ps(kKTdseAng, st);
        k_tdse_velocity<<<(t->N + TI - 1) / TI, 256, smem, st>>>(c, t->P, t->eta, t->plan->knl, t->plan->dk,
                                                                 t->L, t->N, A, idx, tau, t->m0);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    rc = grouped_device_call(1, t->plan, counts, DSBT_C128, 0.0, c, out, kws, kws_b, st);
    if (!rc) rc = potential(t, out, out, E, idx, 0.5 * tau, nullptr, 0.0, nullptr, st);
    return rc;
}

struct TdseWs {
    double2* ckpt;     // [nck][L][N]
    double2* seg;      // [K+1][L][N]
    double2* a;
    double2* mu;
    double2* nu;
    double2* lam;
    double2* tmp;
    void* kws;         // DSBT kinetic workspace
    size_t kws_b;
};

// K >= 1: gradient layout with nsteps/K + 1 checkpoints and a K+1 segment;
// K == 0: propagation only (no checkpoint storage).
size_t ws_layout(const dsbt_tdse* t, int nsteps, int K, TdseWs* w, void* base) {
    const size_t sb = a256(state_bytes(t));
    const int nck = (K >= 1) ? nsteps / K + 1 : 0;
    const size_t kws_b = dsbt_workspace_size(t->plan, t->L, DSBT_C128);
    size_t off = 0;
    unsigned char* p = (unsigned char*)(((uintptr_t)base + 255) & ~(uintptr_t)255);
    auto take = [&](size_t b) { unsigned char* q = p + off; off += a256(b); return q; };
    double2* ck = (double2*)take(sb * nck);
    double2* sg = (K >= 1) ? (double2*)take(sb * (K + 1)) : nullptr;
    double2* a = (double2*)take(sb);
    double2* mu = (double2*)take(sb);
    double2* nu = (double2*)take(sb);
    double2* lam = (double2*)take(sb);
    double2* tmp = (double2*)take(sb);
    void* kws = take(kws_b);
    if (w) *w = TdseWs{ck, sg, a, mu, nu, lam, tmp, kws, kws_b};
    return off + 256;
}

}  // namespace
}  // namespace dsbt

using namespace dsbt;

extern "C" int dsbt_tdse_create(const dsbt_plan* plan, int L, double tau, double Z, double a2,
                                dsbt_tdse** out) {
    return dsbt_tdse_create_m(plan, L, 0, tau, Z, a2, out);
}

extern "C" int dsbt_tdse_create_m(const dsbt_plan* plan, int L, int m, double tau, double Z, double a2,
                                  dsbt_tdse** out) {
    DSBT_CHECK_ARG(plan != nullptr && out != nullptr, "dsbt_tdse_create: NULL argument");
    *out = nullptr;
    const int m0 = m < 0 ? -m : m;
    DSBT_CHECK_ARG(L >= 1 && L <= kLMax && m0 + L - 1 <= plan->l_max,
                   "dsbt_tdse_create: L=%d, |m|=%d need L <= 64 and |m| + L - 1 <= l_max", L, m0);
    DSBT_CHECK_ARG(plan->T64 != nullptr, "dsbt_tdse_create: the plan needs DSBT_PLAN_FP64");
    DSBT_CHECK_ARG(isfinite(tau) && isfinite(Z) && a2 > 0.0, "dsbt_tdse_create: bad tau/Z/a2");
    dsbt_tdse* t = new (std::nothrow) dsbt_tdse();
    if (!t) return DSBT_ERR_NOMEM;
    t->plan = plan;
    t->L = L;
    t->m0 = m0;
    t->N = plan->N;
    t->dr = plan->r_max / plan->N;
    t->tau = tau;
    t->Z = Z;
    t->a2 = a2;
    gauss_legendre(L, t->eta_h, t->w_h);
    std::vector<double> Ph;
    if (m0 == 0) angular_matrix(L, t->eta_h, t->w_h, Ph);
    else angular_matrix_m(L, m0, t->eta_h, t->w_h, Ph);
    std::vector<double> Vh(t->N), rh(t->N);
    for (int i = 0; i < t->N; ++i) {
        rh[i] = (i + 0.5) * t->dr;
        Vh[i] = -Z / sqrt(rh[i] * rh[i] + a2);
    }
    bool ok = cudaMalloc((void**)&t->P, Ph.size() * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&t->V, t->N * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&t->rr, t->N * sizeof(double)) == cudaSuccess &&
              cudaMalloc((void**)&t->eta, L * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMemcpy(t->P, Ph.data(), Ph.size() * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->V, Vh.data(), t->N * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->rr, rh.data(), t->N * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(t->eta, t->eta_h.data(), L * sizeof(double), cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        cudaFree(t->P);
        cudaFree(t->V);
        cudaFree(t->rr);
        cudaFree(t->eta);
        delete t;
        set_error("dsbt_tdse_create: device allocation or copy failed");
        return DSBT_ERR_NOMEM;
    }
    *out = t;
    return DSBT_OK;
}

extern "C" int dsbt_tdse_set_potential(dsbt_tdse* t, const double* V, int n) {
    DSBT_CHECK_ARG(t != nullptr && V != nullptr, "dsbt_tdse_set_potential: NULL argument");
    DSBT_CHECK_ARG(n == t->N, "dsbt_tdse_set_potential: %d values for a grid of %d points", n, t->N);
    for (int i = 0; i < n; ++i) DSBT_CHECK_ARG(isfinite(V[i]), "dsbt_tdse_set_potential: V[%d] not finite", i);
    DSBT_CUDA_TRY(cudaMemcpy(t->V, V, n * sizeof(double), cudaMemcpyHostToDevice));
    return DSBT_OK;
}

extern "C" int dsbt_tdse_destroy(dsbt_tdse* t) {
    if (!t) return DSBT_OK;
    cudaDeviceSynchronize();
    cudaFree(t->P);
    cudaFree(t->V);
    cudaFree(t->rr);
    cudaFree(t->eta);
    delete t;
    return DSBT_OK;
}

extern "C" int dsbt_tdse_angular(const dsbt_tdse* t, double* eta, double* w, double* P) {
    DSBT_CHECK_ARG(t != nullptr, "dsbt_tdse_angular: NULL tdse");
    if (eta) for (int j = 0; j < t->L; ++j) eta[j] = t->eta_h[j];
    if (w) for (int j = 0; j < t->L; ++j) w[j] = t->w_h[j];
    if (P) DSBT_CUDA_TRY(cudaMemcpy(P, t->P, (size_t)t->L * t->L * sizeof(double), cudaMemcpyDeviceToHost));
    return DSBT_OK;
}

extern "C" size_t dsbt_tdse_workspace_size(const dsbt_tdse* t, int nsteps, int checkpoint_every) {
    if (!t || nsteps < 0 || checkpoint_every < 0) return 0;
    return ws_layout(t, nsteps, checkpoint_every, nullptr, nullptr);
}

static int check_run(const dsbt_tdse* t, const void* psi, const double* E, int nsteps, int hold, void* ws,
                     size_t ws_b, int K) {
    DSBT_CHECK_ARG(t != nullptr && psi != nullptr, "tdse: NULL argument");
    DSBT_CHECK_ARG(nsteps >= 0 && hold >= 1, "tdse: nsteps >= 0 and hold >= 1 required");
    DSBT_CHECK_ARG(nsteps == 0 || E != nullptr, "tdse: field samples E is NULL");
    DSBT_CHECK_ARG(ws != nullptr && ws_b >= dsbt_tdse_workspace_size(t, nsteps, K),
                   "tdse: workspace too small (need %zu bytes)", dsbt_tdse_workspace_size(t, nsteps, K));
    return DSBT_OK;
}

extern "C" int dsbt_tdse_propagate(const dsbt_tdse* t, void* psi, const double* E, int nsteps, int hold,
                                   double tau_sign, void* workspace, size_t workspace_bytes, void* stream) {
    int rc = check_run(t, psi, E, nsteps, hold, workspace, workspace_bytes, 0);
    if (rc) return rc;
    DSBT_CHECK_ARG(tau_sign == 1.0 || tau_sign == -1.0, "tdse: tau_sign must be +1 or -1");
    cudaStream_t st = (cudaStream_t)stream;
    TdseWs w;
    ws_layout(t, nsteps, 0, &w, workspace);
    std::vector<int> counts(t->plan->l_max + 1, 0);
    for (int l = 0; l < t->L; ++l) counts[t->m0 + l] = 1;
    double2* x = (double2*)psi;
    const double tau = tau_sign * t->tau;
    for (int s = 0; s < nsteps; ++s) {
        // forward in time: sample s / hold; backward (tau < 0): the samples in reverse
        const int eidx = (tau_sign > 0) ? s / hold : (nsteps - 1 - s) / hold;
        rc = step(t, x, w.a, w.tmp, E, eidx, tau, counts.data(), w.kws, w.kws_b, st);
        if (rc) return rc;
        DSBT_CUDA_TRY(cudaMemcpyAsync(x, w.a, state_bytes(t), cudaMemcpyDeviceToDevice, st));
    }
    return DSBT_OK;
}

extern "C" int dsbt_tdse_propagate_velocity(const dsbt_tdse* t, void* psi, const double* E, const double* A,
                                            int nsteps, int hold, double tau_sign, void* workspace,
                                            size_t workspace_bytes, void* stream) {
    DSBT_CHECK_ARG(t != nullptr && psi != nullptr, "tdse: NULL argument");
    DSBT_CHECK_ARG(nsteps >= 0 && hold >= 1, "tdse: nsteps >= 0 and hold >= 1 required");
    DSBT_CHECK_ARG(workspace != nullptr && workspace_bytes >= dsbt_tdse_workspace_size(t, nsteps, 0),
                   "tdse: workspace too small (need %zu bytes)", dsbt_tdse_workspace_size(t, nsteps, 0));
    DSBT_CHECK_ARG(tau_sign == 1.0 || tau_sign == -1.0, "tdse: tau_sign must be +1 or -1");
    cudaStream_t st = (cudaStream_t)stream;
    TdseWs w;
    ws_layout(t, nsteps, 0, &w, workspace);
    std::vector<int> counts(t->plan->l_max + 1, 0);
    for (int l = 0; l < t->L; ++l) counts[t->m0 + l] = 1;
    double2* x = (double2*)psi;
    const double tau = tau_sign * t->tau;
    for (int s = 0; s < nsteps; ++s) {
        const int idx = (tau_sign > 0) ? s / hold : (nsteps - 1 - s) / hold;
        int rc = step_velocity(t, x, w.a, w.tmp, w.mu, E, A, idx, tau, counts.data(), w.kws, w.kws_b, st);
        if (rc) return rc;
        DSBT_CUDA_TRY(cudaMemcpyAsync(x, w.a, state_bytes(t), cudaMemcpyDeviceToDevice, st));
    }
    return DSBT_OK;
}

extern "C" int dsbt_tdse_observable(const dsbt_tdse* t, const void* psi, double r_cut, double* out,
                                    void* stream) {
    DSBT_CHECK_ARG(t != nullptr && psi != nullptr && out != nullptr, "tdse: NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    DSBT_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), st));
    return observable(t, (const double2*)psi, nullptr, r_cut, out, st);
}

extern "C" int dsbt_tdse_gradient(const dsbt_tdse* t, const void* psi0, const double* E, int nsamples,
                                  int nsteps, int hold, double r_cut, int checkpoint_every, double* O,
                                  double* dOdE, void* workspace, size_t workspace_bytes, void* stream) {
    const int K = checkpoint_every;
    DSBT_CHECK_ARG(K >= 1, "tdse: checkpoint_every must be >= 1");
    int rc = check_run(t, psi0, E, nsteps, hold, workspace, workspace_bytes, K);
    if (rc) return rc;
    DSBT_CHECK_ARG(O != nullptr && dOdE != nullptr, "tdse: NULL output");
    DSBT_CHECK_ARG(nsamples >= (nsteps + hold - 1) / hold, "tdse: nsamples < ceil(nsteps / hold)");
    cudaStream_t st = (cudaStream_t)stream;
    TdseWs w;
    ws_layout(t, nsteps, K, &w, workspace);
    const size_t sb = state_bytes(t);
    const size_t sstride = a256(sb) / sizeof(double2);
    std::vector<int> counts(t->plan->l_max + 1, 0);
    for (int l = 0; l < t->L; ++l) counts[t->m0 + l] = 1;
    const double tau = t->tau;
    // forward sweep with checkpoints every K steps
    DSBT_CUDA_TRY(cudaMemcpyAsync(w.ckpt, psi0, sb, cudaMemcpyDeviceToDevice, st));
    DSBT_CUDA_TRY(cudaMemcpyAsync(w.lam, psi0, sb, cudaMemcpyDeviceToDevice, st));
    for (int s = 0; s < nsteps; ++s) {
        rc = step(t, w.lam, w.a, w.tmp, E, s / hold, tau, counts.data(), w.kws, w.kws_b, st);
        if (rc) return rc;
        std::swap(w.lam, w.a);
        if ((s + 1) % K == 0)
            DSBT_CUDA_TRY(cudaMemcpyAsync(w.ckpt + (size_t)((s + 1) / K) * sstride, w.lam, sb,
                                          cudaMemcpyDeviceToDevice, st));
    }
    // observable and final adjoint state lambda_S = Pi psi_S
    DSBT_CUDA_TRY(cudaMemsetAsync(O, 0, sizeof(double), st));
    rc = observable(t, w.lam, w.mu, r_cut, O, st);
    if (rc) return rc;
    std::swap(w.lam, w.mu);
    DSBT_CUDA_TRY(cudaMemsetAsync(dOdE, 0, (size_t)nsamples * sizeof(double), st));
    // backward sweep, one checkpoint segment at a time
    const int nseg = (nsteps + K - 1) / K;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int s0 = seg * K, s1 = (s0 + K < nsteps) ? s0 + K : nsteps;
        DSBT_CUDA_TRY(cudaMemcpyAsync(w.seg, w.ckpt + (size_t)seg * sstride, sb, cudaMemcpyDeviceToDevice, st));
        for (int s = s0; s < s1; ++s) {
            rc = step(t, w.seg + (size_t)(s - s0) * sstride, w.seg + (size_t)(s - s0 + 1) * sstride, w.tmp, E,
                      s / hold, tau, counts.data(), w.kws, w.kws_b, st);
            if (rc) return rc;
        }
        for (int s = s1 - 1; s >= s0; --s) {
            const double2* psi_s = w.seg + (size_t)(s - s0) * sstride;
            const double2* psi_s1 = w.seg + (size_t)(s - s0 + 1) * sstride;
            double* g = dOdE + s / hold;
            // a_s = Q_s psi_s
            rc = potential(t, psi_s, w.a, E, s / hold, 0.5 * tau, nullptr, 0.0, nullptr, st);
            // mu = Q_s^H lambda_{s+1};  dO/dE += tau Im <lambda_{s+1}, R psi_{s+1}>
            if (!rc) rc = potential(t, w.lam, w.mu, E, s / hold, -0.5 * tau, psi_s1, tau, g, st);
            // nu = Kin^H mu
            if (!rc)
                rc = kinetic_grouped_with_scratch(t->plan, counts.data(), DSBT_C128, -tau, w.mu, w.nu, w.kws,
                                                  w.kws_b, st);
            // lambda_s = Q_s^H nu;  dO/dE += tau Im <nu, R a_s>
            if (!rc) rc = potential(t, w.nu, w.lam, E, s / hold, -0.5 * tau, w.a, tau, g, st);
            if (rc) return rc;
        }
    }
    return DSBT_OK;
}
