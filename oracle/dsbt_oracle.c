/*
 * dsbt_oracle.c -- plain, slow reference implementation of the orthogonal
 * discrete spherical Bessel transform (DSBT) of V. V. Serov,
 * "Orthogonal fast spherical Bessel transform on uniform grid" (arXiv:1509.07115).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link or call this
 * file; it exists so that tests, the smoke check and the CPU-baseline leg of the
 * benchmark can compare the CUDA path against an implementation that follows
 * the paper's definitions step by step.  It shares no code, header or table with
 * the CUDA sources.
 *
 * What it computes (all in FP64 unless stated):
 *   - the discrete Legendre orthogonal polynomials (DLOP) P_l(x, M) by the
 *     three-term recurrence in the degree (Hahn polynomials with alpha=beta=0),
 *     evaluated in IEEE binary128 (_Float128) and rounded to FP64 at the end,
 *     because that recurrence amplifies rounding errors near the grid ends when
 *     the degree approaches M (Sec. 2.3);
 *   - the Fourier matrix F_l (Sec. 2.2, Eq. (16) csFourierBasis), i.e. the
 *     orthonormal DST-II (even l) / DCT-II (odd l) on the midpoint grid, with
 *     each entry's angle reduced exactly in integer arithmetic before sin/cos;
 *   - the Fourier-to-Bessel matrix T_l (Sec. 2.4, Eqs. (38) Tdef, (39) Ldef,
 *     (41) orthoImL, (42) alpha_n; Sec. 2.5, Eq. (43) Tadd);
 *   - forward b = T_l F_l psi and inverse psi = F_l^T T_l^T b (Eqs. (18), (24),
 *     (25)) by naive O(N^2) sums in a fixed order.
 *
 * Index convention: for angular momentum l, p_l = [1+(-1)^l]/2 and the
 * momentum index runs over n = p_l .. N_l = N + p_l - 1 (Eq. (17) k_grid);
 * arrays store it at position n - p_l in [0, N).  Radial samples psi_i,
 * i = 1..N, are stored at position i - 1.
 *
 * Readings of the paper taken here (the printed text is ambiguous there):
 *   - F normalisation: sqrt((2 - delta_{n0})/N) for odd l and
 *     sqrt((2 - delta_{nN})/N) for even l, which makes F orthogonal (the printed
 *     1/sqrt((2 - delta_{n0})N) is not orthogonal);
 *   - F uses plain sin / cos (second line of Eq. (16)); the output then
 *     approximates s_l c_l(k_n) sqrt(w_n) with s_l = (-1)^{ceil(l/2)};
 *   - theta(0) = 1/2 on the diagonal of L (Eq. (11) step_func), which gives the
 *     diagonal of I - L equal to 2 / (1 + P_l(-1, 2n-1));
 *   - the extra rows are n in [p_l, n0_l - 1] (the index range of Eq. (43)).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef _Float128 quad;

/* ---------------------------------------------------------------- helpers */

static int parity_p(int l) { return (l % 2 == 0) ? 1 : 0; }      /* p_l          */
static int n0_of(int l) { return (l + 2) / 2; }                   /* ceil((l+1)/2) */

/* Trapezoid weight factor sqrt(1 - delta_{m0}/2) of Eq. (39) Ldef / Eq. (20). */
static double sqrt_w(long m) { return m == 0 ? sqrt(0.5) : 1.0; }

/*
 * DLOP P_j(x, M), j = 0..lmax, on the points x = 0..M (Sec. 2.3, Eq. (27)
 * DLOPortho with P_j(0, M) = 1).  These are the Hahn polynomials
 * Q_j(x; 0, 0, M), generated by the three-term recurrence in the degree
 *    Q_0 = 1,  Q_1 = 1 - 2x/M,
 *    A_j Q_{j+1} = (A_j + C_j - x) Q_j - C_j Q_{j-1},
 *    A_j = (j+1)(M-j) / (2(2j+1)),  C_j = j(j+M+1) / (2(2j+1)).
 * Only degrees j <= M exist (A_j vanishes at j = M); the caller respects that.
 * x may lie outside [0, M] (x = -1 is used by the tests).
 */
static void dlop_degrees_q(int lmax, long M, long x, quad* out)
{
    quad q0 = 1, q1, xq = (quad)x, Mq = (quad)M;
    out[0] = q0;
    if (lmax == 0) return;
    q1 = 1 - 2 * xq / Mq;
    out[1] = q1;
    for (int j = 1; j < lmax; ++j) {
        quad jq = (quad)j;
        quad A = (jq + 1) * (Mq - jq) / (2 * (2 * jq + 1));
        quad C = jq * (jq + Mq + 1) / (2 * (2 * jq + 1));
        quad q2 = ((A + C - xq) * q1 - C * q0) / A;
        out[j + 1] = q2;
        q0 = q1;
        q1 = q2;
    }
}

static quad dlop_q(int l, long M, long x)
{
    quad buf[130];
    quad* b = buf;
    if (l + 1 > 130) b = (quad*)malloc(sizeof(quad) * (size_t)(l + 1));
    dlop_degrees_q(l, M, x, b);
    quad v = b[l];
    if (b != buf) free(b);
    return v;
}

/* DLOP value rounded to FP64. */
double orc_dlop(int l, long M, long x) { return (double)dlop_q(l, M, x); }

/* Norm factor N(l, M) = (M+l+1)^{falling l+1} / ((2l+1) M^{falling l}),
 * Sec. 2.3, Eq. (28) DLOPnormfac; evaluated as a product of ratios in quad. */
double orc_dlop_norm(int l, long M)
{
    quad v = (quad)(M + l + 1) / (quad)(2 * l + 1);
    for (int j = 1; j <= l; ++j) v *= (quad)(M + l + 1 - j) / (quad)(M - j + 1);
    return (double)v;
}

/* DDLOP P'_l(i, M) = 2 / (1 + P_l(-1, M-1)) * [P_l(i, M-1) - P_l(i-1, M-1)],
 * Sec. 2.3, Eqs. (34)-(35) (backDiff). */
double orc_ddlop(int l, long M, long i)
{
    quad pm1 = dlop_q(l, M - 1, -1);
    quad d = dlop_q(l, M - 1, i) - dlop_q(l, M - 1, i - 1);
    return (double)(2 / (1 + pm1) * d);
}

/* ------------------------------------------------------------ T_l rows */

/*
 * One row of T_l, written at out[m - p], m = p..N_l (Sec. 2.4, 2.5).
 *
 * Regular rows n >= n0_l (Eqs. (38) Tdef, (39) Ldef, (42)):
 *   (I - L)_{nm} = P'_l(n-m, 2n) sqrt(w_m)               for m < n,
 *   (I - L)_{nn} = 1 + P'_l(0, 2n)/2 = 2 / (1 + P_l(-1, 2n-1)),
 *   zero for m > n.  All entries share the positive factor
 *   2 / (1 + P_l(-1, 2n-1)), so the row equals that factor times
 *   u_m = [P_l(n-m, 2n-1) - P_l(n-m-1, 2n-1)] sqrt(w_m) (m < n),  u_n = 1,
 *   and T_{n.} = alpha_n (I - L)_{n.} = u / ||u||_2 with alpha_n of Eq. (42).
 *   Dividing out the common factor avoids forming 1 + P_l(-1, .) - P_l(-1, .).
 *
 * Extra rows p_l <= n < n0_l (Eq. (43) Tadd):
 *   T_{nm} = alpha_n P_{2n-p}(N_l - m, 2 N_l) sqrt(w_m),
 *   alpha_n = sqrt(2 / N(2n-p, 2 N_l))  (closed form stated after Eq. (44)).
 */
static void t_row(int N, int l, long n, double* out)
{
    const int p = parity_p(l);
    const long Nl = (long)N + p - 1;
    const int n0 = n0_of(l);
    memset(out, 0, sizeof(double) * (size_t)N);
    if (n >= n0) {
        const long M = 2 * n - 1;
        const long npts = n - p + 1;                 /* x = 0 .. n - p */
        quad* P = (quad*)malloc(sizeof(quad) * (size_t)npts);
        quad* deg = (quad*)malloc(sizeof(quad) * (size_t)(l + 1));
        for (long x = 0; x < npts; ++x) {
            dlop_degrees_q(l, M, x, deg);
            P[x] = deg[l];
        }
        quad* u = (quad*)malloc(sizeof(quad) * (size_t)npts);
        quad ss = 0;
        for (long m = p; m <= n; ++m) {
            quad v;
            if (m == n) v = 1;
            else {
                long i = n - m;                      /* 1 .. n - p */
                v = (P[i] - P[i - 1]) * (quad)sqrt_w(m);
            }
            u[m - p] = v;
            ss += v * v;
        }
        double nrm = sqrt((double)ss);
        for (long m = p; m <= n; ++m) out[m - p] = (double)(u[m - p] / (quad)nrm);
        free(u);
        free(deg);
        free(P);
    } else {
        const int deg_l = (int)(2 * n - p);
        const long M = 2 * Nl;
        const double alpha = sqrt(2.0 / orc_dlop_norm(deg_l, M));
        quad* deg = (quad*)malloc(sizeof(quad) * (size_t)(deg_l + 1));
        for (long m = p; m <= Nl; ++m) {
            dlop_degrees_q(deg_l, M, Nl - m, deg);
            out[m - p] = alpha * (double)deg[deg_l] * sqrt_w(m);
        }
        free(deg);
    }
}

/* Selected rows of T_l: rows[k] is a storage index n - p in [0, N).
 * out is [nrows][N] row-major.  Returns 0, or -1 on a bad argument. */
int orc_T_rows(int N, int l, int nrows, const int* rows, double* out)
{
    if (N < 2 || l < 0 || 2 * n0_of(l) > 2 * N) return -1;
    const int p = parity_p(l);
    for (int k = 0; k < nrows; ++k) {
        if (rows[k] < 0 || rows[k] >= N) return -1;
        t_row(N, l, (long)rows[k] + p, out + (size_t)k * N);
    }
    return 0;
}

/* Full T_l, [N][N] row-major, entry (n - p, m - p). */
int orc_T_matrix(int N, int l, double* T)
{
    if (N < 2 || l < 0 || n0_of(l) > N) return -1;
    const int p = parity_p(l);
    for (int r = 0; r < N; ++r) t_row(N, l, (long)r + p, T + (size_t)r * N);
    return 0;
}

/* ------------------------------------------------------------ F_l */

/*
 * F_l (Sec. 2.2, Eq. (16) csFourierBasis with Eqs. (14) r_grid, (17) k_grid):
 *   k_n r_i = n (i - 1/2) pi / N.
 *   even l: F_{ni} = sqrt((2 - delta_{nN})/N) sin(pi n (2i-1) / (2N)), n = 1..N
 *   odd  l: F_{ni} = sqrt((2 - delta_{n0})/N) cos(pi n (2i-1) / (2N)), n = 0..N-1
 * The integer n(2i-1) is reduced modulo 4N before the angle is formed, so the
 * argument passed to sin/cos lies in [0, 2 pi).
 */
static double f_entry(int N, int l, long n, long i)
{
    const long a = (n * (2 * i - 1)) % (4L * N);
    const double ang = M_PI * (double)a / (2.0 * (double)N);
    if (l % 2 == 0) {
        const double c = (n == N) ? sqrt(1.0 / N) : sqrt(2.0 / N);
        return c * sin(ang);
    } else {
        const double c = (n == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
        return c * cos(ang);
    }
}

int orc_F_matrix(int N, int l, double* F)
{
    if (N < 2 || l < 0) return -1;
    const int p = parity_p(l);
    for (int r = 0; r < N; ++r)
        for (int c = 0; c < N; ++c) F[(size_t)r * N + c] = f_entry(N, l, (long)r + p, (long)c + 1);
    return 0;
}

/* ------------------------------------------------------------ transforms */

/*
 * Forward DSBT of nlines real lines: b = T_l (F_l psi) (Eqs. (18), (24)).
 * psi, b: [nlines][N].  Both matrices are formed explicitly, then applied by
 * naive sums over the column index in increasing order.
 */
int orc_forward(int N, int l, int nlines, const double* psi, double* b)
{
    if (N < 2 || l < 0 || n0_of(l) > N || nlines < 0) return -1;
    double* F = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* T = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* f = (double*)malloc(sizeof(double) * (size_t)N);
    orc_F_matrix(N, l, F);
    orc_T_matrix(N, l, T);
    for (int c = 0; c < nlines; ++c) {
        const double* x = psi + (size_t)c * N;
        for (int r = 0; r < N; ++r) {
            double s = 0;
            for (int i = 0; i < N; ++i) s += F[(size_t)r * N + i] * x[i];
            f[r] = s;
        }
        for (int r = 0; r < N; ++r) {
            double s = 0;
            for (int m = 0; m < N; ++m) s += T[(size_t)r * N + m] * f[m];
            b[(size_t)c * N + r] = s;
        }
    }
    free(f);
    free(T);
    free(F);
    return 0;
}

/* Inverse DSBT: psi = F_l^T (T_l^T b) (Eq. (25) with T^{-1} = T^T). */
int orc_inverse(int N, int l, int nlines, const double* b, double* psi)
{
    if (N < 2 || l < 0 || n0_of(l) > N || nlines < 0) return -1;
    double* F = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* T = (double*)malloc(sizeof(double) * (size_t)N * N);
    double* f = (double*)malloc(sizeof(double) * (size_t)N);
    orc_F_matrix(N, l, F);
    orc_T_matrix(N, l, T);
    for (int c = 0; c < nlines; ++c) {
        const double* y = b + (size_t)c * N;
        for (int m = 0; m < N; ++m) {
            double s = 0;
            for (int r = 0; r < N; ++r) s += T[(size_t)r * N + m] * y[r];
            f[m] = s;
        }
        for (int i = 0; i < N; ++i) {
            double s = 0;
            for (int r = 0; r < N; ++r) s += F[(size_t)r * N + i] * f[r];
            psi[(size_t)c * N + i] = s;
        }
    }
    free(f);
    free(T);
    free(F);
    return 0;
}

/*
 * Apply a given explicit matrix (row-major [N][N]) or its transpose to nlines
 * real lines by naive sums.  Used to apply F_l and T_l when the caller already
 * holds them (sampled checks at large N).
 */
int orc_apply(int N, const double* A, int transpose, int nlines, const double* x, double* y)
{
    if (N < 1 || nlines < 0) return -1;
    for (int c = 0; c < nlines; ++c) {
        const double* xc = x + (size_t)c * N;
        for (int r = 0; r < N; ++r) {
            double s = 0;
            if (!transpose)
                for (int k = 0; k < N; ++k) s += A[(size_t)r * N + k] * xc[k];
            else
                for (int k = 0; k < N; ++k) s += A[(size_t)k * N + r] * xc[k];
            y[(size_t)c * N + r] = s;
        }
    }
    return 0;
}
