// eigen.cu -- bound states of one l channel by imaginary-time evolution
// (Sec. 4.4): the paper substitutes t -> -i t in the split-step propagator and
// orthogonalises every state against the lower ones after each step.
//
// One step on nstates real FP64 states psi[s][i] (channel l, spherical
// potential U(r_i)):
//   psi *= exp(-U tau/2);  b = T_l F_l psi;  b *= exp(-k^2 tau/2);
//   psi = F_l^T T_l^T b;   psi *= exp(-U tau/2);
//   modified Gram-Schmidt over s (R_ss = the norm before normalising).
// This is orthogonal iteration with S = exp(-U tau/2) B^T exp(-K tau) B
// exp(-U tau/2), so state s converges to S's s-th eigenvector and
// -ln(R_ss)/tau to its level.  The momenta are the plan's (dsbt_plan_get_k).
#include <math.h>

#include <vector>

#include "plan.cuh"

namespace dsbt {


namespace {

constexpr int kThreads = 1024;

// psi[s][i] *= exp(-U_i ht)
__global__ void k_eig_potential(double* psi, const double* __restrict__ U, int N, int ns, double ht) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)ns * N) return;
    psi[k] *= exp(-U[k % N] * ht);
}

// b[s][j] *= exp(-k_j^2 ht) with the plan's momenta of channel l
__global__ void k_eig_kinetic(double* b, const double* __restrict__ knl, double dk, int l, int N, int ns,
                              double ht) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (long long)ns * N) return;
    const int j = (int)(k % N);
    const double km = knl ? knl[(size_t)l * N + j] : k_index(l, j, N) * dk;
    b[k] *= exp(-km * km * ht);
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (lane < (int)(blockDim.x >> 5)) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[32] = v;
    }
    __syncthreads();
    return red[32];
}

// Modified Gram-Schmidt of the ns states (one CTA); rdiag[s] = norm of state s
// after removing the lower states, before normalising.
__global__ void __launch_bounds__(kThreads) k_eig_orthonormalise(double* psi, int N, int ns, double* rdiag) {
    __shared__ double red[33];
    for (int s = 0; s < ns; ++s) {
        double* x = psi + (size_t)s * N;
        for (int t = 0; t < s; ++t) {
            const double* y = psi + (size_t)t * N;
            double d = 0.0;
            for (int i = threadIdx.x; i < N; i += blockDim.x) d = fma(x[i], y[i], d);
            d = block_sum(d, red);
            for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] = fma(-d, y[i], x[i]);
            __syncthreads();
        }
        double q = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) q = fma(x[i], x[i], q);
        q = block_sum(q, red);
        const double nrm = sqrt(q);
        if (threadIdx.x == 0) rdiag[s] = nrm;
        const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) x[i] *= inv;
        __syncthreads();
    }
}

// E[s] = sum_j (k_j^2/2) b[s][j]^2 + sum_i U_i psi[s][i]^2 for normalised psi.
__global__ void __launch_bounds__(kThreads) k_eig_energy(const double* __restrict__ psi,
                                                         const double* __restrict__ b,
                                                         const double* __restrict__ U,
                                                         const double* __restrict__ knl, double dk, int l,
                                                         int N, double* E) {
    __shared__ double red[33];
    const int s = blockIdx.x;
    double e = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double km = knl ? knl[(size_t)l * N + i] : k_index(l, i, N) * dk;
        const double bv = b[(size_t)s * N + i], pv = psi[(size_t)s * N + i];
        e += 0.5 * km * km * bv * bv + U[i] * pv * pv;
    }
    e = block_sum(e, red);
    if (threadIdx.x == 0) E[s] = e;
}

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace dsbt

using namespace dsbt;

extern "C" size_t dsbt_radial_states_workspace_size(const dsbt_plan* plan, int nstates) {
    if (!plan || nstates < 1 || nstates > 64) return 0;
    return a256((size_t)nstates * plan->N * sizeof(double)) + a256(3 * 64 * sizeof(double)) +
           dsbt_workspace_size(plan, nstates, DSBT_F64) + 512;
}

extern "C" int dsbt_radial_states(const dsbt_plan* plan, int l, const double* U, int nstates, double tau,
                                  int nsteps, double* psi, double* levels, double* energies, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    DSBT_CHECK_ARG(plan != nullptr && U != nullptr && psi != nullptr, "dsbt_radial_states: NULL argument");
    DSBT_CHECK_ARG(plan->T64 != nullptr, "dsbt_radial_states: the plan needs DSBT_PLAN_FP64");
    DSBT_CHECK_ARG(l >= 0 && l <= plan->l_max, "dsbt_radial_states: l=%d outside 0..%d", l, plan->l_max);
    DSBT_CHECK_ARG(nstates >= 1 && nstates <= 64, "dsbt_radial_states: nstates=%d not in 1..64", nstates);
    DSBT_CHECK_ARG(tau > 0.0 && isfinite(tau), "dsbt_radial_states: tau must be positive");
    DSBT_CHECK_ARG(nsteps >= 1, "dsbt_radial_states: nsteps must be >= 1");
    const size_t need = dsbt_radial_states_workspace_size(plan, nstates);
    DSBT_CHECK_ARG(workspace != nullptr && workspace_bytes >= need,
                   "dsbt_radial_states: workspace too small (need %zu bytes)", need);
    cudaStream_t st = (cudaStream_t)stream;
    const int N = plan->N, ns = nstates;
    unsigned char* base = (unsigned char*)(((uintptr_t)workspace + 255) & ~(uintptr_t)255);
    double* b = (double*)base;
    double* small = (double*)(base + a256((size_t)ns * N * sizeof(double)));   // rdiag, E
    void* gws = base + a256((size_t)ns * N * sizeof(double)) + a256(3 * 64 * sizeof(double));
    const size_t gws_b = dsbt_workspace_size(plan, ns, DSBT_F64);
    std::vector<int> counts(plan->l_max + 1, 0);
    counts[l] = ns;
    const long long tot = (long long)ns * N;
    const unsigned g = (unsigned)((tot + 255) / 256);
    int rc;
    {
        ProfScope ps(kKTdseReduce, st);
        k_eig_orthonormalise<<<1, kThreads, 0, st>>>(psi, N, ns, small);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    for (int step = 0; step < nsteps; ++step) {
        {
            ProfScope ps(kKTdsePot, st);
            k_eig_potential<<<g, 256, 0, st>>>(psi, U, N, ns, 0.5 * tau);
        }
        rc = grouped_device_call(0, plan, counts.data(), DSBT_F64, 0.0, psi, b, gws, gws_b, st);
        if (rc) return rc;
        {
            ProfScope ps(kKPhase, st);
            k_eig_kinetic<<<g, 256, 0, st>>>(b, plan->knl, plan->dk, l, N, ns, 0.5 * tau);
        }
        rc = grouped_device_call(1, plan, counts.data(), DSBT_F64, 0.0, b, psi, gws, gws_b, st);
        if (rc) return rc;
        {
            ProfScope ps(kKTdsePot, st);
            k_eig_potential<<<g, 256, 0, st>>>(psi, U, N, ns, 0.5 * tau);
        }
        {
            ProfScope ps(kKTdseReduce, st);
            k_eig_orthonormalise<<<1, kThreads, 0, st>>>(psi, N, ns, small);
        }
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    // energies <psi|H|psi> of the final (normalised) states
    rc = grouped_device_call(0, plan, counts.data(), DSBT_F64, 0.0, psi, b, gws, gws_b, st);
    if (rc) return rc;
    {
        ProfScope ps(kKTdseReduce, st);
        k_eig_energy<<<ns, kThreads, 0, st>>>(psi, b, U, plan->knl, plan->dk, l, N, small + 64);
        DSBT_CUDA_TRY(cudaGetLastError());
    }
    std::vector<double> h(128);
    DSBT_CUDA_TRY(cudaMemcpyAsync(h.data(), small, 128 * sizeof(double), cudaMemcpyDeviceToHost, st));
    DSBT_CUDA_TRY(cudaStreamSynchronize(st));
    for (int s = 0; s < ns; ++s) {
        if (levels) levels[s] = -log(h[s]) / tau;
        if (energies) energies[s] = h[64 + s];
    }
    return DSBT_OK;
}
