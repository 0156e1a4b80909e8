// kcorr.cu -- corrected momenta k_nl (Sec. 3, Eq. (kcorr)) for the kinetic
// phase of plans built with DSBT_PLAN_KCORR.
//
// The paper asks for the momentum at which the Riccati-Bessel function
// chi_l(x) = x j_l(x) meets the DSBT basis function's boundary condition at
// r_max: chi_l(k r_max) = 0 (even l), chi_l'(k r_max) = 0 (odd l).  Coefficient
// n of a regular row (n >= n0_l) takes the m-th positive root, m = n -
// floor(l/2): the basis function near r_max goes like sin(k_n r - l pi/2), so
// it has made as many half-waves as chi_l at its m-th zero.  Completion rows
// take the largest grid momentum N dk, as in the uniform grid (k_index).
//
// Method (host, FP64).  Write chi_l = M sin(theta), -x y_l(x) = M cos(theta).
// The phase theta(x) rises monotonically from 0 with theta' = 1/M^2 (the
// Wronskian), so the m-th zero of chi_l is the solution of theta(x) = m pi,
// found by Newton's method on theta inside a bracket that is kept from the
// previous zero.  For odd l the zero of chi_l' in the m-th lobe (between zeros
// m-1 and m of chi_l, where chi_l has exactly one extremum) is found by Newton's
// method on chi_l' with chi_l'' = (l(l+1)/x^2 - 1) chi_l, again bracketed.
// j_l comes from upward recurrence for x > l and from normalised downward
// recurrence below; y_l from upward recurrence.  The theta branch is fixed with
// the WKB phase sqrt(x^2 - nu^2) - nu acos(nu/x) + pi/4 (nu = l + 1/2) beyond
// the turning point, where it is accurate to far better than pi.
#include <math.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "plan.cuh"

namespace dsbt {

namespace {

struct JY {
    double j, jm1, y;   // j_l(x), j_{l-1}(x) (0 for l = 0), y_l(x)
};

JY bessel(int l, double x) {
    const double s = sin(x), c = cos(x);
    JY r;
    // y_l upward (stable for every x)
    double y0 = -c / x, y1 = -c / (x * x) - s / x;
    if (l == 0) {
        r.y = y0;
    } else {
        for (int k = 1; k < l; ++k) {
            const double y2 = (2 * k + 1) / x * y1 - y0;
            y0 = y1;
            y1 = y2;
        }
        r.y = y1;
    }
    const double j0 = s / x, j1 = s / (x * x) - c / x;
    if (l == 0) {
        r.j = j0;
        r.jm1 = 0.0;
        return r;
    }
    if (x > l) {   // upward
        double a = j0, b = j1;
        for (int k = 1; k < l; ++k) {
            const double t = (2 * k + 1) / x * b - a;
            a = b;
            b = t;
        }
        r.j = b;
        r.jm1 = a;
        return r;
    }
    // downward from well above l, normalised by j_0 or j_1 (whichever is larger)
    const int start = l + 40 + (int)x;
    double up = 0.0, cur = 1e-300, jl = 0.0, jlm1 = 0.0, f0 = 0.0, f1 = 0.0;
    for (int k = start; k >= 1; --k) {   // cur = f_k, up = f_{k+1}; f_{k-1} = (2k+1)/x f_k - f_{k+1}
        const double down = (2 * k + 1) / x * cur - up;
        up = cur;
        cur = down;
        if (k - 1 == l) jl = cur;
        if (k - 1 == l - 1) jlm1 = cur;
        if (k - 1 == 1) f1 = cur;
        if (k - 1 == 0) f0 = cur;
        if (fabs(cur) > 1e250) {   // rescale
            up *= 1e-250;
            cur *= 1e-250;
            jl *= 1e-250;
            jlm1 *= 1e-250;
            f1 *= 1e-250;
        }
    }
    const double scale = (fabs(j0) > fabs(j1)) ? j0 / f0 : j1 / f1;
    r.j = jl * scale;
    r.jm1 = jlm1 * scale;
    return r;
}

struct Phase {
    double theta, M2, chi, dchi;
};

Phase phase(int l, double x) {
    const JY b = bessel(l, x);
    Phase p;
    const double a = x * b.j, c = -x * b.y;
    p.chi = a;
    // chi' = j_l + x j_l' with j_l' = j_{l-1} - (l+1)/x j_l  (j_0' = -j_1)
    const double djl = (l == 0) ? -(sin(x) / (x * x) - cos(x) / x) : b.jm1 - (l + 1) / x * b.j;
    p.dchi = b.j + x * djl;
    p.M2 = a * a + c * c;
    double th = atan2(a, c);
    const double nu = l + 0.5;
    if (x > nu) {
        const double wkb = sqrt(x * x - nu * nu) - nu * acos(nu / x) + M_PI / 4;
        th += 2 * M_PI * nearbyint((wkb - th) / (2 * M_PI));
    }
    p.theta = th;
    return p;
}

// Zero of f on (lo, hi) (f(lo), f(hi) of opposite signs) by Newton steps with
// bisection whenever a step leaves the bracket.
template <typename F>
double bracketed_newton(F f, double lo, double hi, double x0) {
    double flo = f(lo).first;
    double x = std::min(std::max(x0, lo), hi);
    for (int it = 0; it < 200; ++it) {
        const std::pair<double, double> v = f(x);   // value, derivative
        if (v.first == 0.0) return x;
        if ((v.first < 0) == (flo < 0)) {
            lo = x;
            flo = v.first;
        } else {
            hi = x;
        }
        double xn = (v.second != 0.0) ? x - v.first / v.second : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 4e-16 * fabs(x) || hi - lo <= 4e-16 * hi) return xn;
        x = xn;
    }
    return x;
}

void fill_l(int N, double r_max, int l, double* out) {
    const double dk = M_PI / r_max;
    const int p = parity_p(l), n0 = n0_of(l), half = l / 2;
    for (int s = 0; s < N; ++s) out[s] = k_index(l, s, N) * dk;
    const int m_last = (N - 1 + p) - half;
    if (m_last < 1) return;
    // zeros of chi_l: theta(x) = m pi, m = 1..m_last
    std::vector<double> z(m_last + 1, 0.0);
    double prev = 1e-3;
    for (int m = 1; m <= m_last; ++m) {
        const double target = m * M_PI;
        const double hi = target + l * M_PI / 2 + 1e-9;   // theta(x) > x - l pi / 2 there
        const double guess = std::max(prev + 1e-9, hi - l * (l + 1) / (2 * hi));
        z[m] = bracketed_newton(
            [&](double x) {
                const Phase ph = phase(l, x);
                return std::make_pair(ph.theta - target, 1.0 / ph.M2);
            },
            prev, hi, guess);
        prev = z[m];
    }
    for (int n = std::max(n0, p); n <= N - 1 + p; ++n) {
        const int m = n - half;
        double x = z[m];
        if (l & 1) {   // zero of chi_l' in lobe m: between zeros m-1 and m of chi_l
            const double lo = (m == 1) ? 1e-3 : z[m - 1];
            const double hi = z[m];
            const double c = l * (l + 1.0);
            x = bracketed_newton(
                [&](double t) {
                    const Phase ph = phase(l, t);
                    return std::make_pair(ph.dchi, (c / (t * t) - 1.0) * ph.chi);
                },
                lo, hi, hi - M_PI / 2);
        }
        out[n - p] = x / r_max;
    }
}

}  // namespace

// Corrected momentum table [(l_max+1)][N] (storage index s = n - p_l).
void kcorr_table(int N, double r_max, int l_max, std::vector<double>& out) {
    out.assign((size_t)(l_max + 1) * N, 0.0);
    const int L = l_max + 1;
    unsigned hw = std::thread::hardware_concurrency();
    const int nthreads = (int)std::max(1u, std::min<unsigned>(hw ? hw : 1u, 16u));
    std::vector<std::thread> pool;
    for (int t = 0; t < nthreads; ++t)
        pool.emplace_back([&, t]() {
            for (int l = t; l < L; l += nthreads) fill_l(N, r_max, l, out.data() + (size_t)l * N);
        });
    for (auto& th : pool) th.join();
}

}  // namespace dsbt

using namespace dsbt;

extern "C" int dsbt_plan_get_k(const dsbt_plan* plan, int l, double* host_out) {
    DSBT_CHECK_ARG(plan != nullptr && host_out != nullptr, "dsbt_plan_get_k: NULL argument");
    DSBT_CHECK_ARG(l >= 0 && l <= plan->l_max, "dsbt_plan_get_k: l=%d outside 0..%d", l, plan->l_max);
    const int N = plan->N;
    if (plan->knl) {
        DSBT_CUDA_TRY(cudaMemcpy(host_out, plan->knl + (size_t)l * N, N * sizeof(double), cudaMemcpyDeviceToHost));
        return DSBT_OK;
    }
    for (int s = 0; s < N; ++s) host_out[s] = k_index(l, s, N) * plan->dk;
    return DSBT_OK;
}
