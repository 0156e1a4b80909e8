/*
 * dsbt.h -- C ABI of the GB300 (sm_103a) orthogonal discrete spherical Bessel
 * transform (DSBT) of V. V. Serov, "Orthogonal fast spherical Bessel transform
 * on uniform grid" (arXiv:1509.07115).
 *
 * The transform of one radial channel of angular momentum l is
 *     b = T_l F_l psi                                   (Sec. 2.2, Eqs. (18), (24))
 * with F_l the orthonormal sine (even l) / cosine (odd l) transform on the
 * midpoint grid (Eq. (16)) and T_l the orthogonal Fourier-to-Bessel matrix
 * built from derivatives of discrete Legendre orthogonal polynomials
 * (Sec. 2.4 Eqs. (38)-(42), completed by the rows of Sec. 2.5 Eq. (43)).
 * The inverse is psi = F_l^T T_l^T b (Eq. (25), T^{-1} = T^T).
 *
 * Data conventions (all arrays are caller-owned DEVICE memory unless stated):
 *   - A channel is N consecutive samples psi_i = psi(r_i) sqrt(dr), i = 1..N,
 *     r_i = (i - 1/2) dr, dr = r_max / N (Eq. (14)); psi = r Psi_lm.
 *   - Output coefficient k of a channel is b_n for n = k + p_l, p_l =
 *     [1 + (-1)^l]/2 (Eq. (17)); b_n approximates s_l c_l(k_n) sqrt(dk) with
 *     k_n = n pi / r_max and s_l = (-1)^{ceil(l/2)} (plain sin/cos in F_l).
 *   - Complex dtypes are interleaved (re, im); channel c starts at element c*N.
 *   - Grouped calls take channels of all l = 0..l_max back to back, l-major:
 *     counts[l] channels of angular momentum l (counts is a HOST array of
 *     l_max + 1 ints; zero counts are allowed).
 *
 * Precision paths:
 *   - DSBT_F64 / DSBT_C128: everything in FP64 (sine/cosine transform by an
 *     FP64 FFT, T_l contraction by FP64 FMA).
 *   - DSBT_F32 / DSBT_C64: FP32 FFT, T_l contraction on the tcgen05 tensor
 *     cores as a compensated split product (T = T_hi + T_lo, x = x_hi + x_lo,
 *     T x ~ T_hi x_hi + T_hi x_lo + T_lo x_hi, FP32 accumulation in TMEM):
 *     TF32 pairs for the dense factors (DSBT_PLAN_TF32X3); FP16 pairs (same
 *     11 significant bits, twice the tensor rate, half the bytes) for the
 *     interval scheme (DSBT_PLAN_FAST_SPLIT), with T_l scaled by 2^14 and each
 *     channel by a power of two 2^e, ||2^e psi|| in [2^12, 2^13), so that no
 *     intermediate leaves the FP16 range; scales are exact and removed before
 *     any FP32 output.
 *
 * Errors: every entry point returns an int status (DSBT_OK = 0, negative on
 * failure) and never throws; dsbt_last_error() returns a thread-local message
 * for the last failure on the calling thread.  Arguments are validated on the
 * host before any launch.  Calls are asynchronous on the given stream
 * (a cudaStream_t passed as void*, NULL = legacy default stream); a plan is
 * immutable after creation and may be shared by several streams, but a
 * workspace must not be used by two calls that overlap in time.
 */
#ifndef DSBT_H
#define DSBT_H

#include <stddef.h>

#if defined(__GNUC__)
#define DSBT_API __attribute__((visibility("default")))
#else
#define DSBT_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define DSBT_OK 0
#define DSBT_ERR_INVALID (-1)     /* bad argument (null pointer, size, l range, dtype) */
#define DSBT_ERR_NOMEM (-2)       /* device allocation failed during plan creation   */
#define DSBT_ERR_PLAN_CHECK (-3)  /* plan failed its orthogonality check             */
#define DSBT_ERR_CUDA (-4)        /* a CUDA runtime call failed                       */
#define DSBT_ERR_TIMEOUT (-5)     /* a device-side wait gave up (see dsbt_device_status) */
#define DSBT_ERR_UNSUPPORTED (-6) /* path not built into this plan / size unsupported */

/* plan flags: which factor copies to build (at least one of the first two) */
#define DSBT_PLAN_FP64 1   /* FP64 T_l (for DSBT_F64 / DSBT_C128 calls)            */
#define DSBT_PLAN_TF32X3 2 /* split-TF32 T_l and T_l^T (for DSBT_F32 / DSBT_C64)  */
#define DSBT_PLAN_KCORR 4  /* kinetic phase with the corrected momenta k_nl (Sec. 3,
                              Eq. (kcorr)) instead of k~_n (see dsbt_plan_get_k) */
#define DSBT_PLAN_FAST64 8 /* with DSBT_PLAN_FP64, N / 64 a power of two: FP64
                              contractions on planar lines (the kinetic step, the
                              TDSE) in O(N l log N) work instead of N^2/2: rows of
                              T_l are polynomials in m left of the diagonal, applied
                              through a tree of interval moments in orthonormal
                              polynomial bases (stable counterpart of Sec. 2.6).
                              Extra memory: 8 B x 64 x (l_max+1) x N x log2(N/64)
                              of plan data; FP64 workspaces grow by about
                              8 B x 128 x (N/64) per line. */
#define DSBT_PLAN_FAST_SPLIT 16 /* any plan grid (N / 128 leaves of 128 rows):
                              split-precision contractions (all DSBT_F32 /
                              DSBT_C64 calls) in O(N l log N) work on the tensor
                              cores: near band of T_l per leaf (diagonal blocks),
                              far field through 64 basis functions per dyadic
                              interval of the column tree (the rows of T_l are
                              polynomials of degree l - 1 in m left of the
                              diagonal, Eqs. (38)-(42)), operands as FP16 pairs.
                              Needs l_max <= 64 (always true); with or without
                              DSBT_PLAN_TF32X3 (whose dense copies it does not
                              use).  Extra memory: about
                              8 B x 64 x (l_max+1) x N x (log2(N/128) + 4) of plan
                              data (1.2 GB at N = 4096, l_max = 63) plus
                              16 B x 64 x N x N/128 for the interval bases, and
                              4 B x 64 x (N/128 + log2(N/128)) per line of
                              workspace (plus one 4-byte counter per 256
                              lines). */
#define DSBT_PLAN_FAST_TF32 DSBT_PLAN_FAST_SPLIT /* earlier name of the same flag */

/* element types of the caller's arrays */
#define DSBT_F64 1  /* real double                 */
#define DSBT_C128 2 /* complex double, interleaved  */
#define DSBT_F32 3  /* real float                  */
#define DSBT_C64 4  /* complex float, interleaved   */

typedef struct dsbt_plan dsbt_plan;

/*
 * Build a plan for grids of N points (256 <= N <= 8192, N a multiple of 256) and
 * angular momenta l = 0..l_max (0 <= l_max <= 64, with ceil((l_max+1)/2) <= N).
 * r_max only sets the momentum step dk = pi / r_max used by the kinetic phase.
 * Runs on the current CUDA device and stream `stream`; returns once the plan is
 * built and has passed its check.  The plan owns every device buffer it
 * allocates (T_l in FP64 and/or split TF32, FFT twiddles); dsbt_plan_destroy
 * frees them.  Factors are generated on the GPU in FP64 (Sec. 2.3-2.5) by the
 * difference equation of the DLOP in x, then each T_l passes a probe check
 * max|T^T (T x) - x| / max|x| <= 1e-12 on random x; failure returns
 * DSBT_ERR_PLAN_CHECK and no plan.
 */
DSBT_API int dsbt_plan_create(int N, double r_max, int l_max, int flags, void* stream, dsbt_plan** out);

/* Release every device buffer of the plan (synchronises the device first).
 * Accepts NULL. */
DSBT_API int dsbt_plan_destroy(dsbt_plan* plan);

/* Plan facts: grid size, l_max, flags, and the largest probe error of the
 * orthogonality check (written to whichever pointers are non-NULL). */
DSBT_API int dsbt_plan_info(const dsbt_plan* plan, int* N, int* l_max, int* flags, double* check_err);

/*
 * Copy T_l (storage index (n - p_l, m - p_l), row-major N x N, FP64) of a plan
 * built with DSBT_PLAN_FP64 into the caller's DEVICE buffer `dst`
 * (N*N doubles).  For inspection and tests.
 */
DSBT_API int dsbt_plan_get_T(const dsbt_plan* plan, int l, double* dst, void* stream);

/*
 * Copy the N momenta that the kinetic phase of this plan uses for angular
 * momentum l (storage index s = n - p_l) into the HOST array host_out.
 * Regular rows n >= n0_l: without DSBT_PLAN_KCORR k~_n = n dk (Eq. (65));
 * with it (Sec. 3, Eq. (kcorr)) k_nl = x_m / r_max with x_m the m-th positive
 * zero (m = n - floor(l/2)) of chi_l(x) = x j_l(x) for even l, of chi_l'(x)
 * for odd l.  Completion rows n < n0_l (n = 0 of odd l among them) take the
 * largest grid momentum N dk in both cases.  The table is computed on the host in FP64 at plan creation
 * (relative accuracy ~1e-16).  Synchronous.
 */
DSBT_API int dsbt_plan_get_k(const dsbt_plan* plan, int l, double* host_out);

/*
 * Bytes of device workspace needed by a call on `total_channels` channels of
 * element type `dtype` (any of the calls below).  The caller allocates it
 * (256-byte aligned) and passes it with its size; its contents need not be
 * initialised and are scratch after the call.
 */
DSBT_API size_t dsbt_workspace_size(const dsbt_plan* plan, int total_channels, int dtype);

/*
 * Forward DSBT of `nchan` channels of one angular momentum l:
 *     out[c] = T_l F_l in[c],  c = 0..nchan-1   (Eqs. (18), (24)).
 * in, out: device arrays of nchan*N elements of `dtype`; they may not overlap.
 */
DSBT_API int dsbt_forward(const dsbt_plan* plan, int l, int nchan, int dtype, const void* in, void* out,
                 void* workspace, size_t workspace_bytes, void* stream);

/* Inverse DSBT: out[c] = F_l^T T_l^T in[c]  (Eq. (25), T^{-1} = T^T). */
DSBT_API int dsbt_inverse(const dsbt_plan* plan, int l, int nchan, int dtype, const void* in, void* out,
                 void* workspace, size_t workspace_bytes, void* stream);

/*
 * Grouped forward / inverse over all l = 0..l_max in one call: counts[l]
 * channels of each l, stored l-major (counts is a HOST array of l_max+1 ints).
 * Same contract as dsbt_forward / dsbt_inverse per group.
 */
DSBT_API int dsbt_forward_grouped(const dsbt_plan* plan, const int* counts, int dtype, const void* in,
                         void* out, void* workspace, size_t workspace_bytes, void* stream);
DSBT_API int dsbt_inverse_grouped(const dsbt_plan* plan, const int* counts, int dtype, const void* in,
                         void* out, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Free-particle kinetic step through the DSBT (the kinetic factor of the
 * split-operator scheme, Sec. 4.1, Eq. (81), with the momentum grid of
 * Eq. (65)): out = F^T T^T exp(-i K tau) T F in, per l group, where
 * K = diag(k_n^2 / 2) with the plan's momenta (dsbt_plan_get_k): k~_n = n dk
 * on the regular rows, N dk on the completion rows n < n0_l (which project
 * onto non-regular high-frequency functions; with n0_l - p_l = 0 rows for
 * l = 0 this is Eq. (65)'s rule that the n = 0 coefficient of odd l takes
 * k~_N).  Complex dtypes only (DSBT_C128, DSBT_C64).
 * The phase is applied inside the forward contraction's epilogue.
 */
DSBT_API int dsbt_kinetic_grouped(const dsbt_plan* plan, const int* counts, int dtype, double tau,
                         const void* in, void* out, void* workspace, size_t workspace_bytes,
                         void* stream);

/*
 * Grouped forward DSBT for callers that cannot allocate device memory (their
 * device memory is owned by a framework allocator, a cudaMalloc's implicit
 * synchronisation is not acceptable in their loop, or their memory budget is
 * fixed at start-up).  The paper has no counterpart: this is a deployment
 * variant of dsbt_forward_grouped with the same arguments and results, minus
 * the workspace.  Its scratch is a static 64 MiB device array that every GPU
 * loading this library reserves until the process exits; a call whose
 * dsbt_workspace_size exceeds 64 MiB (roughly sum(counts) * N > 2^21 complex
 * samples) is rejected with DSBT_ERR_INVALID before any launch.  The call
 * allocates nothing: every call looks up the array's device address with
 * cudaGetSymbolAddress on the current device (no cached address, so the call
 * stays valid after cudaDeviceReset); the first call on a device may load the
 * library's device code there, so make that first call before any stream
 * capture.  All calls on a device share the one array, so calls that may
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The plan must belong to the current device.
 */
DSBT_API int dsbt_forward_grouped_noalloc(const dsbt_plan* plan, const int* counts, int dtype,
                                          const void* in, void* out, void* stream);

/*
 * Grouped transforms of HOST-resident channels (same layouts and results as
 * dsbt_forward_grouped / dsbt_inverse_grouped / dsbt_kinetic_grouped, which
 * see): the channels are cut into nchunks contiguous ranges (0 = 8; clamped to
 * the channel count) and streamed through the GPU so that the host-to-device
 * copy of one chunk, the transform of the previous one and the device-to-host
 * copy of the one before overlap (two internal streams plus `stream`).  host_in
 * and host_out should be pinned (cudaHostAlloc / cudaHostRegister): pageable
 * memory gives the same results without the overlap.  The workspace is a
 * DEVICE buffer of dsbt_host_workspace_size bytes (two input and two output
 * slots of one chunk plus the transform workspace of one chunk).  Asynchronous:
 * work on `stream` issued later runs after host_out is written; the caller
 * synchronises `stream` before reading host_out.  Errors as the device calls,
 * checked before any copy is issued.
 */
DSBT_API size_t dsbt_host_workspace_size(const dsbt_plan* plan, const int* counts, int dtype, int nchunks);
DSBT_API int dsbt_forward_grouped_host(const dsbt_plan* plan, const int* counts, int dtype, const void* host_in,
                                       void* host_out, int nchunks, void* workspace, size_t workspace_bytes,
                                       void* stream);
DSBT_API int dsbt_inverse_grouped_host(const dsbt_plan* plan, const int* counts, int dtype, const void* host_in,
                                       void* host_out, int nchunks, void* workspace, size_t workspace_bytes,
                                       void* stream);
DSBT_API int dsbt_kinetic_grouped_host(const dsbt_plan* plan, const int* counts, int dtype, double tau,
                                       const void* host_in, void* host_out, int nchunks, void* workspace,
                                       size_t workspace_bytes, void* stream);

/*
 * Read the plan's device status word (synchronous: waits for the device).
 * 0 = OK; 1 = a device-side wait in a tensor-core contraction gave up after its
 * iteration limit (the kernel then skipped its remaining work, after letting
 * its own TMA copies and MMAs already in flight finish; the results of that
 * call are undefined, the context and the plan stay usable).  reset != 0
 * clears the word afterwards.
 */
DSBT_API int dsbt_device_status(const dsbt_plan* plan, int reset, int* status_out);

/*
 * Re-run the plan's orthogonality probe (Eq. (25), T^{-1} = T^T) on its FP64
 * factors: max |T^T (T x) - x| over two pseudo-random x per l into *err_out
 * (may be NULL); DSBT_ERR_PLAN_CHECK above 1e-12, DSBT_ERR_UNSUPPORTED for a
 * plan without DSBT_PLAN_FP64.  Synchronous on `stream`.
 */
DSBT_API int dsbt_plan_check(dsbt_plan* plan, double* err_out, void* stream);

/*
 * Testing hooks for the failure paths (no counterpart in the paper).
 * dsbt_plan_set_spin_limit: polls of each bounded mbarrier wait in this plan's
 * tensor-core kernels (0 restores the default, 2^25); a small value makes
 * waits give up, which a later dsbt_device_status reports.
 * dsbt_plan_perturb_T: adds delta to entry (row, col) of the FP64 T_l (not to
 * the split copies), so that dsbt_plan_check sees a corrupt factor.
 * Both change a plan that is otherwise immutable: no call may be in flight on
 * it.  Synchronous.
 */
DSBT_API int dsbt_plan_set_spin_limit(dsbt_plan* plan, unsigned polls);
DSBT_API int dsbt_plan_perturb_T(dsbt_plan* plan, int l, int row, int col, double delta, void* stream);

/*
 * Tile order of the DSBT_PLAN_FAST_SPLIT contraction (a tuning knob; the paper
 * has no counterpart).  Each direction is one launch over "units" (a group's
 * column tile of 256 lines): the unit's moment (forward) or weight (adjoint)
 * tiles, then its row tiles, which read the lines again and the moments just
 * written.  The launch runs unit u's first tiles together with the row tiles
 * of unit u - lag, so the second reading comes from L2; a row tile waits
 * (bounded, on a device counter) until its unit's first tiles are stored.
 * lag >= 1; a lag at least the number of units is the plain order (every
 * first tile, then every row tile), the default: on a GB300 at N = 4096,
 * l <= 63 the longest moment tiles run for tens of microseconds, so row tiles
 * at short lags wait and the units between them outgrow L2 (lag 16 measured
 * 12 % slower than the plain order).  Results do not depend on the lag: every
 * tile computes the same sums in the same order.  DSBT_ERR_INVALID for lag < 1,
 * DSBT_ERR_UNSUPPORTED for a plan without DSBT_PLAN_FAST_SPLIT.  No call may be
 * in flight on the plan.
 */
DSBT_API int dsbt_plan_set_fast_lag(dsbt_plan* plan, int lag);

/* ---------------------------------------------------------------------------
 * Bound states of one l channel (Sec. 4.4): imaginary-time evolution with the
 * split propagator S = exp(-U tau/2) F^T T^T exp(-K tau) T F exp(-U tau/2)
 * (K = k^2/2 with the plan's momenta, see dsbt_plan_get_k) and, after every
 * step, modified Gram-Schmidt of each state against the lower ones.
 * U: DEVICE array of N potential values U(r_i) (midpoint grid, spherical
 * potential); psi: DEVICE array [nstates][N] of real FP64 radial states
 * (psi(r_i) sqrt(dr)), in: a starting guess with a component along every
 * wanted state, out: the normalised states after nsteps steps.  levels (HOST,
 * nstates, may be NULL): -ln(R_ss)/tau with R_ss the norm of state s after one
 * step and the projection (the levels of S that the states converge to);
 * energies (HOST, may be NULL): <psi_s| F^T T^T K T F + U |psi_s> of the
 * final states.  Plan built with DSBT_PLAN_FP64; 1 <= nstates <= 64;
 * workspace: DEVICE, dsbt_radial_states_workspace_size bytes.  Synchronises
 * the stream before returning (the outputs are on the host).
 * ------------------------------------------------------------------------- */
DSBT_API size_t dsbt_radial_states_workspace_size(const dsbt_plan* plan, int nstates);
DSBT_API int dsbt_radial_states(const dsbt_plan* plan, int l, const double* U, int nstates, double tau,
                                int nsteps, double* psi, double* levels, double* energies, void* workspace,
                                size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Split-operator TDSE through the DSBT (Sec. 4.1, Eq. (81)) for an axially
 * symmetric state (m = 0) in a linearly polarised field in the length gauge
 * (vector potential A = 0):  H = p^2/2 + V(r) + E(t) r cos(theta),
 * V(r) = -Z / sqrt(r^2 + a2).  The state is psi[l][i] (complex128, l = 0..L-1,
 * i = 0..N-1, radial samples as for the DSBT) in the l representation.  One
 * step of length tau:  psi <- Q Kin Q psi  with
 *   Q   = P diag(exp(-i [V(r_i) + E r_i eta_j] tau/2)) P^T on the L-point
 *         Gauss-Legendre grid eta_j (P[l][j] = sqrt((2l+1)/2) P_l(eta_j) sqrt(w_j)),
 *   Kin = the kinetic step of dsbt_kinetic_grouped (one channel per l).
 * Step s uses the field sample E[s / hold] (a DEVICE array of doubles).
 * ------------------------------------------------------------------------- */
typedef struct dsbt_tdse dsbt_tdse;

/* Propagator over a plan built with DSBT_PLAN_FP64 and l_max >= L-1 (L <= 64);
 * the plan must outlive it.  Owns small device tables (P, V, r, eta). */
DSBT_API int dsbt_tdse_create(const dsbt_plan* plan, int L, double tau, double Z, double a2,
                              dsbt_tdse** out);
/* The same for a state of fixed magnetic quantum number m (an axially
 * symmetric potential and a field along z conserve m): channels
 * l = |m| .. |m| + L - 1 (the plan needs l_max >= |m| + L - 1), angular
 * transform P[i][j] = the normalised associated Legendre functions
 * Pbar_{|m|+i}^{|m|}(eta_j) sqrt(w_j), orthonormalised on the L-point
 * Gauss-Legendre rule by Gram-Schmidt in order of l (Sec. 4.1: associated
 * Legendre functions orthonormalised on the quadrature).  m = 0 is
 * dsbt_tdse_create.  Every dsbt_tdse_* call then works on [L][N] states of
 * those channels. */
DSBT_API int dsbt_tdse_create_m(const dsbt_plan* plan, int L, int m, double tau, double Z, double a2,
                                dsbt_tdse** out);
DSBT_API int dsbt_tdse_destroy(dsbt_tdse* tdse);

/*
 * Velocity-gauge steps (Eq. (81) with the vector potential A(t) along z):
 * psi <- exp(-iU tau/2) Y^T B^T exp(-iK tau/2) Ytilde exp(i A k~_n eta tau)
 *        Ytilde^dagger exp(-iK tau/2) B Y exp(-iU tau/2) psi,
 * U = V(r) + E r eta as in dsbt_tdse_propagate (E may be NULL: no length-gauge
 * field), A[s / hold] the vector-potential sample of step s (DEVICE array,
 * NULL: A = 0), Ytilde the angular transform with the i^l factors of the
 * modified spherical harmonics taken on the momentum grid k~_n = n dk.  The
 * kinetic half phases use the plan's momenta (dsbt_plan_get_k).  Workspace as
 * dsbt_tdse_workspace_size(tdse, nsteps, 0).  tau_sign = -1 runs the inverse
 * steps with the samples in reverse.
 */
DSBT_API int dsbt_tdse_propagate_velocity(const dsbt_tdse* tdse, void* psi, const double* E, const double* A,
                                          int nsteps, int hold, double tau_sign, void* workspace,
                                          size_t workspace_bytes, void* stream);

/* Replace the radial potential V(r_i) (the soft-Coulomb default of
 * dsbt_tdse_create) with the caller's n = N HOST values on the midpoint grid
 * r_i = (i + 1/2) dr, i = 0..N-1.  Synchronous. */
DSBT_API int dsbt_tdse_set_potential(dsbt_tdse* tdse, const double* V, int n);

/* Host copies of the angular grid: eta[L], w[L] and P[L*L] (any may be NULL). */
DSBT_API int dsbt_tdse_angular(const dsbt_tdse* tdse, double* eta, double* w, double* P);

/* Device workspace for dsbt_tdse_propagate (checkpoint_every = 0: five states
 * of L*N complex128 plus one DSBT workspace) or for dsbt_tdse_gradient with
 * nsteps steps and a checkpoint every K >= 1 steps (nsteps/K + K + 7 states
 * plus one DSBT workspace). */
DSBT_API size_t dsbt_tdse_workspace_size(const dsbt_tdse* tdse, int nsteps, int checkpoint_every);

/* Propagate psi (device, in place) by nsteps steps.  tau_sign = +1 steps
 * forward; tau_sign = -1 applies the inverse steps (tau -> -tau) with the field
 * samples walked backwards, so a forward run followed by a backward run returns
 * the initial state (unitarity, Eq. (25)). */
DSBT_API int dsbt_tdse_propagate(const dsbt_tdse* tdse, void* psi, const double* E, int nsteps,
                                 int hold, double tau_sign, void* workspace, size_t workspace_bytes,
                                 void* stream);

/* *out (device double) = sum over r_i > r_cut and all l of |psi[l][i]|^2. */
DSBT_API int dsbt_tdse_observable(const dsbt_tdse* tdse, const void* psi, double r_cut, double* out,
                                  void* stream);

/*
 * Gradient of O = sum_{r_i > r_cut} |psi_S|^2 (psi_S = state after nsteps from
 * psi0, which is not modified) with respect to the nsamples field samples E,
 * by the adjoint method: forward sweep storing a checkpoint every
 * checkpoint_every steps, then a backward sweep that recomputes each segment
 * from its checkpoint and runs the adjoint step (the same step with tau ->
 * -tau, since P and T_l are orthogonal).  Writes O (device double) and dOdE
 * (device array of nsamples doubles).
 */
DSBT_API int dsbt_tdse_gradient(const dsbt_tdse* tdse, const void* psi0, const double* E, int nsamples,
                                int nsteps, int hold, double r_cut, int checkpoint_every, double* O,
                                double* dOdE, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * The full DSBT-DVR step (Sec. 4.1): all magnetic quantum numbers at once, for
 * potentials and fields without axial symmetry.  Channels (l, m) with
 * m = -M .. M and, for each m, l = |m| .. |m| + L - 1 (the fixed-m ranges of
 * dsbt_tdse_create_m, so the angular transform is square per m), stored
 * l-major as psi[c][i] (complex128, i = 0..N-1); dsbt_tdse3d_channels lists
 * (l, m) per channel c.  Angular grid: L Gauss-Legendre nodes eta_j = cos(theta_j)
 * times NM = 2M + 1 angles phi_q = 2 pi q / NM; Y = P Phi with P^m as in
 * dsbt_tdse_create_m and Phi[m][q] = exp(i m phi_q) / sqrt(NM) (Sec. 4.1, the
 * DFT over phi), unitary on the channel space.  One step of length tau:
 *   psi <- Q Kin Q psi,  Q = Y^H diag(exp(-i [V(r) + r F.n] tau/2)) Y,
 *   n = (sin theta cos phi, sin theta sin phi, cos theta),
 *   Kin = the kinetic step of dsbt_kinetic_grouped (each channel with its l),
 * with F = (F[3s'], F[3s'+1], F[3s'+2]), s' = s / hold, the field sample of step
 * s (a DEVICE array; NULL: no field).  V defaults to 0.  A field along z couples
 * no m and reproduces dsbt_tdse_create_m for every m.
 * ------------------------------------------------------------------------- */
typedef struct dsbt_tdse3d dsbt_tdse3d;

/* Plan built with DSBT_PLAN_FP64 and l_max >= M + L - 1; 1 <= L <= 32,
 * 0 <= M <= 12.  The plan must outlive the propagator.  Errors: -1 on bad
 * arguments (or too much shared memory for L, M), -3 out of memory. */
DSBT_API int dsbt_tdse3d_create(const dsbt_plan* plan, int L, int M, double tau, dsbt_tdse3d** out);
DSBT_API int dsbt_tdse3d_destroy(dsbt_tdse3d* tdse);
/* *nchan and, per channel c, l_of[c] and m_of[c] (HOST arrays of nchan ints, may be NULL). */
DSBT_API int dsbt_tdse3d_channels(const dsbt_tdse3d* tdse, int* nchan, int* l_of, int* m_of);
/* The radial potential V(r_i) from n = N HOST values on the midpoint grid.  Synchronous. */
DSBT_API int dsbt_tdse3d_set_potential(dsbt_tdse3d* tdse, const double* V, int n);
/* Device workspace: two states plus one DSBT workspace. */
DSBT_API size_t dsbt_tdse3d_workspace_size(const dsbt_tdse3d* tdse);
/* Propagate psi (device, in place) by nsteps steps, asynchronous on stream. */
DSBT_API int dsbt_tdse3d_propagate(const dsbt_tdse3d* tdse, void* psi, const double* F, int nsteps, int hold,
                                   void* workspace, size_t workspace_bytes, void* stream);
/* Velocity-gauge steps (Eq. (81)) with the vector potential A of any direction:
 * psi <- exp(-iU tau/2) Y^H B^T exp(-iK tau/2) Ytilde exp(i k~_n (A.n) tau)
 *        Ytilde^H exp(-iK tau/2) B Y exp(-iU tau/2) psi,
 * U = V(r) + r F.n (F may be NULL), A = (A[3s'], A[3s'+1], A[3s'+2]), s' = s / hold
 * (DEVICE array, NULL: A = 0), Ytilde = Y with the factors i^l of the modified
 * harmonics on the momentum grid k~_n = n dk; the kinetic half phases use the
 * plan's momenta.  Same workspace as dsbt_tdse3d_propagate. */
DSBT_API int dsbt_tdse3d_propagate_velocity(const dsbt_tdse3d* tdse, void* psi, const double* F, const double* A,
                                            int nsteps, int hold, void* workspace, size_t workspace_bytes,
                                            void* stream);

/*
 * Gradient of O = sum over r_i > r_cut and all channels of |psi_S|^2 (psi_S the
 * state after nsteps length-gauge steps of dsbt_tdse3d_propagate from psi0,
 * which is not modified) with respect to the 3 x nsamples field components F
 * (same layout as in dsbt_tdse3d_propagate), by the adjoint method: a forward
 * sweep storing a checkpoint every checkpoint_every steps, then a backward
 * sweep that recomputes each segment and runs the adjoint step (the same step
 * with tau -> -tau, Y and T_l being unitary / orthogonal), accumulating
 * tau Im <Y lambda, r n_c Y psi> in the angular kernel (n the direction of the
 * angular node).  Writes O (device double) and dOdF (device [nsamples][3]).
 * The paper has no gradient; this extends its propagator (Sec. 4.1).
 */
DSBT_API size_t dsbt_tdse3d_gradient_workspace_size(const dsbt_tdse3d* tdse, int nsteps, int checkpoint_every);
DSBT_API int dsbt_tdse3d_gradient(const dsbt_tdse3d* tdse, const void* psi0, const double* F, int nsamples,
                                  int nsteps, int hold, double r_cut, int checkpoint_every, double* O,
                                  double* dOdF, void* workspace, size_t workspace_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batch of uneven transforms (different grids and l_max) sharing one factor
 * set.  The regular rows of T_l (Sec. 2.4) do not depend on the grid size N;
 * only the completion rows (Sec. 2.5, Eq. (43)) do.  A batch builds the
 * split-TF32 factors once at (N_max, max l_max) plus, per distinct N, a table of
 * the first 32 rows, and runs the contraction of every transform in one
 * persistent launch per direction.  Complex64 data only.
 *
 * Layout of the caller's batch arrays: transforms t = 0..ntrans-1 back to back;
 * transform t holds sum_l counts_t[l] channels of N[t] complex samples, l-major.
 * counts is the concatenation of the per-transform count arrays (l_max[t] + 1
 * entries each).  All transforms share the radial step dr (r_max_t = N[t] dr).
 * ------------------------------------------------------------------------- */
typedef struct dsbt_batch dsbt_batch;

/* N[t] a multiple of 256 in [256, 8192], 0 <= l_max[t] <= 64.  The batch owns
 * its factors, tables, workspace and tensor maps (about
 * 16 B (max l_max + 1) N_max^2 + 16 B per complex sample of the batch).  With
 * autotune_tiles != 0 it times the contraction's tile order (see
 * dsbt_batch_set_tiles) and column-tile width (128/192/256 lines) on its own
 * shapes and keeps the fastest; otherwise it takes order 3 at width 256.
 * Synchronises the stream. */
DSBT_API int dsbt_batch_create(int ntrans, const int* N, const int* l_max, const int* counts, double dr,
                               int autotune_tiles, void* stream, dsbt_batch** out);

/* dsbt_batch_create with flags: DSBT_BATCH_AUTOTUNE (as autotune_tiles above)
 * and DSBT_BATCH_INTERVAL: instead of the shared dense factors and the
 * persistent launch, one DSBT_PLAN_FAST_SPLIT plan per distinct grid (l_max
 * the largest of the transforms on that grid), and per grid one grouped call
 * on its plan (the O(N l log N) interval scheme) over the channels of every
 * transform on that grid, which the sine/cosine kernels gather from and
 * scatter back to the batch arrays through a table of channel offsets; the
 * grids' calls are spread over four internal streams that fork from and join
 * back into the caller's stream, and dsbt_batch_capture_kinetic captures the
 * whole fork-join graph.  Plan data about 8 B x 64 x (l_max+1) x N x
 * (log2(N/128) + 4) per distinct grid plus a workspace per internal stream.
 * On such a batch dsbt_batch_info reports order -1 and width 0, and
 * dsbt_batch_set_tiles is unsupported.  Same results as the dense batch
 * within the split-precision bar. */
#define DSBT_BATCH_AUTOTUNE 1
#define DSBT_BATCH_INTERVAL 2
DSBT_API int dsbt_batch_create_ex(int ntrans, const int* N, const int* l_max, const int* counts, double dr,
                                  int flags, void* stream, dsbt_batch** out);
DSBT_API int dsbt_batch_destroy(dsbt_batch* batch);

/* Complex elements of one batch array, the chosen tile order and width, and
 * the twelve autotuner timings in ms (order-major, widths 128/192/256; zero
 * when the batch was created without autotuning). */
DSBT_API int dsbt_batch_info(const dsbt_batch* batch, long long* total_elems, int* order, int* bn_cap,
                             float* tune_ms);

/* Host-only planning check (no device is touched): builds the forward and
 * inverse tile lists the batch described by (ntrans, N, l_max, counts) would
 * use at (order, bn_cap), checks them against the kernel's rules, and returns
 * their lengths and the forward list's B-operand lines (segments x 32; the
 * padding overhead is seg_lines / real lines).  DSBT_ERR_INVALID for bad
 * arguments or a list that breaks a rule.  NULL outputs are skipped. */
DSBT_API int dsbt_batch_tiles(int ntrans, const int* N, const int* l_max, const int* counts, int order, int bn_cap,
                              int* ntiles_fwd, int* ntiles_inv, long long* seg_lines);

/* Pin the contraction's tile order and column-tile width (128, 192 or 256
 * lines), overriding the autotuner.  Orders: 0 transform-major, 1 l-major
 * (each (transform, l) group's tiles together), 2 l-major with row tiles
 * interleaved across the transforms of one l, 3 as 2 with 32-line segments of
 * different transforms packed into one tile.  DSBT_ERR_INVALID for other
 * values.  Results do not depend on the tiling except through FP32 rounding
 * order.  Graphs captured earlier stay valid and keep their own tiling.
 * Synchronises the stream. */
DSBT_API int dsbt_batch_set_tiles(dsbt_batch* batch, int order, int bn_cap, void* stream);

/* Forward DSBT of every channel of the batch (DEVICE arrays, complex64). */
DSBT_API int dsbt_batch_forward(const dsbt_batch* batch, const void* in, void* out, void* stream);

/* Kinetic step (as dsbt_kinetic_grouped, with k~_n = n pi / (N_t dr) per
 * transform) of every channel of the batch. */
DSBT_API int dsbt_batch_kinetic(const dsbt_batch* batch, double tau, const void* in, void* out, void* stream);

/* Capture dsbt_batch_kinetic(batch, tau, in, out) into an executable CUDA
 * graph (after one uncaptured run); replay it with dsbt_graph_launch on any
 * stream, free it with dsbt_graph_destroy.  The graph keeps the pointers in
 * and out: replays read and write those buffers. */
DSBT_API int dsbt_batch_capture_kinetic(const dsbt_batch* batch, double tau, const void* in, void* out,
                                        void** graph_exec);
DSBT_API int dsbt_graph_launch(void* graph_exec, void* stream);
DSBT_API int dsbt_graph_destroy(void* graph_exec);

/*
 * Launch accounting and kernel timing (tracing).  dsbt_launch_count returns the
 * number of kernel launches the library has issued in this process.
 * dsbt_profile_enable(1) clears earlier records and starts recording a pair of
 * CUDA events on the launch stream around every kernel launch (0 stops);
 * dsbt_profile_read synchronises on the recorded events of one kernel kind and
 * returns how many launches were recorded and their summed device time in ms.
 * dsbt_kernel_name maps a kernel id (0, 1, ...) to its name, NULL past the last.
 */
DSBT_API long long dsbt_launch_count(void);
DSBT_API int dsbt_profile_enable(int on);
DSBT_API int dsbt_profile_read(int kernel_id, int* launches, double* total_ms);
DSBT_API const char* dsbt_kernel_name(int kernel_id);

/* Thread-local text of the last error on this thread ("" if none). */
DSBT_API const char* dsbt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* DSBT_H */
