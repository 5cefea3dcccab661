// C ABI of libgfc: argument checks, node tables, per-stream scratch, and the
// launch sequence of one evaluation (G0(mu2) first, then the points).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "gfc.h"
#include "gfc_df.h"

#include <nvtx3/nvToolsExt.h>
#include "gfc_internal.h"

namespace gfc {

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;
static thread_local gfc_eval_stats g_last_stats;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int fail(int code, const char *msg) { return fail(code, std::string(msg)); }

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(GFC_ECUDA, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                               cudaGetErrorString(e) + ")");
}

// test hook: the next g_fail_allocs device allocations fail (host-side fault
// injection; the GPU is never faulted)
static std::atomic<int> g_fail_allocs{0};

static bool take_injected_failure()
{
    int v = g_fail_allocs.load();
    while (v > 0 && !g_fail_allocs.compare_exchange_weak(v, v - 1)) {
    }
    return v > 0;
}

cudaError_t dev_malloc(void **p, size_t bytes)
{
    if (take_injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s)
{
    if (take_injected_failure()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, s);
}

// test hook: the next g_fail_launches evaluation launches report an error
// without launching anything
static std::atomic<int> g_fail_launches{0};

bool take_injected_launch_failure()
{
    int v = g_fail_launches.load();
    while (v > 0 && !g_fail_launches.compare_exchange_weak(v, v - 1)) {
    }
    return v > 0;
}

// test switch: evaluate every node over the full angular table (no
// compressed rules)
static std::atomic<int> g_full_rule{0};

bool full_rule_forced() { return g_full_rule.load() != 0; }

// NVTX range for the duration of one ABI call (a no-op without a tool)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

// ---------------------------------------------------------------------------
// Gauss-Legendre rule on [-1, 1] (Abramowitz & Stegun 25.4.29), computed by
// Newton's method on f(theta) = P_n(cos theta) in the angle variable: the
// nodes are x = cos theta and the weights 2 / f'(theta)^2, so 1 - x^2 never
// has to be formed near the ends of the interval.
// ---------------------------------------------------------------------------
static void legendre_and_derivative(int n, double x, double &p, double &dp)
{
    double p0 = 1.0, p1 = x;
    if (n == 0) {
        p = 1.0;
        dp = 0.0;
        return;
    }
    for (int k = 2; k <= n; ++k) {
        double pk = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = pk;
    }
    p = p1;
    // P_n'(x) (1 - x^2) = n (P_(n-1)(x) - x P_n(x))
    dp = n * (p0 - x * p1);   // = (1 - x^2) P_n'(x)
}

void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        // root i counted from the right end: theta in (0, pi/2]
        double th = pi * (i + 0.75) / (n + 0.5);
        for (int it = 0; it < 60; ++it) {
            double c = std::cos(th), s = std::sin(th), p, q;
            legendre_and_derivative(n, c, p, q);
            // d/dtheta P_n(cos theta) = -sin(theta) P_n'(cos theta) = -q / s
            double d = -q / s;
            double step = p / d;
            th -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double c = std::cos(th), s = std::sin(th), p, q;
        legendre_and_derivative(n, c, p, q);
        double d = q / s;                     // |f'(theta)|
        double wi = 2.0 / (d * d);
        x[n - 1 - i] = c;
        w[n - 1 - i] = wi;
        x[i] = -c;
        w[i] = wi;
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

// ---------------------------------------------------------------------------
// node tables (per device, cached by rule)
// ---------------------------------------------------------------------------
struct Tables {
    int n_r, n_a, dim, ang_rule;
    double L;
    double2 *rad64 = nullptr, *seg64 = nullptr, *arc64 = nullptr;
    double2 *rayp64 = nullptr;   // (rho^2, rho^(D-1) W) of the radial nodes
    float4 *rayq_df = nullptr;   // double-float (rho^2 s, s), (rho^(D-1) W s^3), s = 1/(1 + rho^2)
    float2 *rad32 = nullptr, *seg32 = nullptr, *arc32 = nullptr;
    float4 *rad_df = nullptr, *seg_df = nullptr, *arc_df = nullptr;
    double2 *tail64 = nullptr;
    float2 *tail32 = nullptr;
    float4 *tail_df = nullptr;
    double *ang64 = nullptr;
    float *ang32 = nullptr;
    float2 *ang_df = nullptr;
    float2 *rules_df = nullptr;
    std::vector<double> t, e, g;
    double Omega = 0, Omega1 = 0, delta = 0;
    // compressed angular rules
    int nrule = 0;
    int rule_off[kMaxRules] = {}, rule_n[kMaxRules] = {};
    float rho_min32[kMaxRules] = {}, rho_min64[kMaxRules] = {};
    double *rules64 = nullptr;
    float4 *rules32 = nullptr;
    int rules_total = 0;
    size_t bytes = 0;
};

// ---------------------------------------------------------------------------
// Compressed angular rules. For a fixed point and radial node the pair sum is
// T2(w) = sum_j e_j / (1 - w t_j), a Stieltjes sum of the discrete measure
// mu = sum_j e_j delta(t - t_j) on [0, 1]. The n-point Gauss rule of mu
// (nodes tau_k, weights gamma_k) integrates polynomials of degree < 2n exactly,
// so for f(t) = 1/(1 - w t), analytic inside the Bernstein ellipse through the
// pole t = 1/w, it reproduces T2 with relative error ~ rho^(-2n), rho the
// ellipse parameter of 2/w - 1. The recurrence coefficients of mu come from
// Lanczos on diag(t) with the start vector sqrt(e) (full reorthogonalisation);
// the rule's nodes are the eigenvalues of the resulting Jacobi matrix and its
// weights the Christoffel numbers (gauss_from_jacobi).
// ---------------------------------------------------------------------------

// Solves T x = r in place for the tridiagonal T (sub-diagonal l[1..n),
// diagonal d, super-diagonal u[0..n-1)) by Gaussian elimination with partial
// pivoting (a row swap fills one extra super-diagonal). A zero pivot is
// replaced by `tiny`: the inverse iteration below solves with a T that is
// singular to working precision on purpose.
static void tri_solve(int n, const std::vector<double> &l, const std::vector<double> &d,
                      const std::vector<double> &u, double tiny, std::vector<double> &r)
{
    std::vector<double> a(n), b(n, 0.0), c(n, 0.0);
    // the row being eliminated, entries at columns (i, i+1, i+2) and its right side
    double p0 = d[0], p1 = n > 1 ? u[0] : 0.0, p2 = 0.0, pr = r[0];
    for (int i = 0; i + 1 < n; ++i) {
        double q0 = l[i + 1], q1 = d[i + 1], q2 = i + 2 < n ? u[i + 1] : 0.0, qr = r[i + 1];
        if (std::fabs(q0) > std::fabs(p0)) {
            std::swap(p0, q0);
            std::swap(p1, q1);
            std::swap(p2, q2);
            std::swap(pr, qr);
        }
        if (p0 == 0.0) p0 = tiny;
        const double m = q0 / p0;
        a[i] = p0;
        b[i] = p1;
        c[i] = p2;
        r[i] = pr;
        p0 = q1 - m * p1;
        p1 = q2 - m * p2;
        p2 = 0.0;
        pr = qr - m * pr;
    }
    a[n - 1] = p0 == 0.0 ? tiny : p0;
    r[n - 1] = pr;
    for (int i = n - 1; i >= 0; --i) {
        double s = r[i];
        if (i + 1 < n) s -= b[i] * r[i + 1];
        if (i + 2 < n) s -= c[i] * r[i + 2];
        r[i] = s / a[i];
    }
}

// K of the compressed rules' thresholds rho_min(n) = exp(K / n): the n-node
// rule's relative error ~ 10 rho^(-2n) stays below 2^-52 (binary64 and
// double-float nodes) or 2^-26 (binary32) for rho >= rho_min(n)
static const double kRuleK64 = 0.5 * std::log(10.0 * std::pow(2.0, 52));
static const double kRuleK32 = 0.5 * std::log(10.0 * std::pow(2.0, 26));

// Gauss rule of order n from the Jacobi matrix J of a measure of mass mu0
// (diagonal a[0..n), off-diagonal b[0..n-1), b > 0). Nodes: the eigenvalues
// of J, each found by bisection on the Sturm count (the number of negative
// pivots of the LDL^T factorisation of J - lambda I equals the number of
// eigenvalues below lambda). Weights: mu0 v_0^2 for the unit eigenvector v,
// found by inverse iteration with the converged eigenvalue (Golub-Welsch).
// Returns false if a weight is not finite and positive.
static bool gauss_from_jacobi(int n, const std::vector<double> &a, const std::vector<double> &b,
                              double mu0, std::vector<double> &nodes, std::vector<double> &weights)
{
    // Gershgorin interval holding every eigenvalue
    double lo = a[0], hi = a[0];
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(b[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    // eigenvalues of J strictly below lam
    auto count_below = [&](double lam) {
        int c = 0;
        double d = 1.0;
        for (int i = 0; i < n; ++i) {
            d = (a[i] - lam) - (i > 0 ? b[i - 1] * (b[i - 1] / d) : 0.0);
            if (d == 0.0) d = -1e-300;   // a zero pivot: perturb lam infinitesimally
            if (d < 0.0) ++c;
        }
        return c;
    };
    const double tiny = 1e-30 * std::max(std::fabs(lo), std::fabs(hi));
    std::vector<double> sub(n, 0.0), dg(n), sup(n, 0.0), v(n);
    for (int i = 0; i + 1 < n; ++i) {
        sub[i + 1] = b[i];
        sup[i] = b[i];
    }
    nodes.assign(n, 0.0);
    weights.assign(n, 0.0);
    for (int k = 0; k < n; ++k) {
        // the k-th eigenvalue (ascending) lies where the count passes k
        double l = lo, h = hi;
        for (int it = 0; it < 200; ++it) {
            const double m = 0.5 * (l + h);
            if (!(m > l && m < h)) break;
            if (count_below(m) > k) h = m;
            else l = m;
        }
        const double lam = 0.5 * (l + h);
        nodes[k] = lam;
        for (int i = 0; i < n; ++i) {
            dg[i] = a[i] - lam;
            v[i] = 1.0;
        }
        for (int it = 0; it < 3; ++it) {
            tri_solve(n, sub, dg, sup, tiny, v);
            double s = 0.0;
            for (double x : v) s = std::max(s, std::fabs(x));
            for (double &x : v) x /= s;
        }
        double s2 = 0.0;
        for (double x : v) s2 += x * x;
        weights[k] = mu0 * v[0] * v[0] / s2;
        if (!(weights[k] > 0.0) || !std::isfinite(weights[k])) return false;
    }
    return true;
}

static void build_rules(Tables &T, std::vector<double> &r64, std::vector<float4> &r32)
{
    const int N = (int)T.t.size();
    // sizes spaced by at most ~12 %, so that the smallest exact rule of a node
    // over-provisions little
    static const int cand[] = {2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 16, 18, 20, 22,
                               24, 27, 30, 33, 36, 40, 44, 48, 53, 58, 64, 70, 77, 85, 96};
    std::vector<int> ns;
    for (int n : cand)
        if (n < N && (int)ns.size() < kMaxRules) ns.push_back(n);
    T.nrule = 0;
    T.rules_total = 0;
    if (ns.empty()) return;
    const int nmax = ns.back();
    // Lanczos on diag(t) from q0 = sqrt(e)/|sqrt(e)|
    double mu0 = 0.0;
    for (double v : T.e) mu0 += v;
    std::vector<std::vector<double>> Q(nmax + 1, std::vector<double>(N, 0.0));
    double nrm = 0.0;
    for (int j = 0; j < N; ++j) nrm += T.e[j];
    nrm = std::sqrt(nrm);
    for (int j = 0; j < N; ++j) Q[0][j] = std::sqrt(T.e[j]) / nrm;
    std::vector<double> alpha(nmax, 0.0), beta(nmax, 0.0);
    int kmax = nmax;
    for (int k = 0; k < nmax; ++k) {
        std::vector<double> v(N);
        for (int j = 0; j < N; ++j) v[j] = T.t[j] * Q[k][j];
        double a = 0.0;
        for (int j = 0; j < N; ++j) a += Q[k][j] * v[j];
        alpha[k] = a;
        for (int j = 0; j < N; ++j) v[j] -= a * Q[k][j] + (k > 0 ? beta[k - 1] * Q[k - 1][j] : 0.0);
        for (int pass = 0; pass < 2; ++pass)
            for (int i = 0; i <= k; ++i) {
                double h = 0.0;
                for (int j = 0; j < N; ++j) h += Q[i][j] * v[j];
                for (int j = 0; j < N; ++j) v[j] -= h * Q[i][j];
            }
        double b = 0.0;
        for (int j = 0; j < N; ++j) b += v[j] * v[j];
        b = std::sqrt(b);
        beta[k] = b;
        if (b < 1e-14) {
            kmax = k + 1;
            break;
        }
        for (int j = 0; j < N; ++j) Q[k + 1][j] = v[j] / b;
    }
    // thresholds: relative error ~ 10 rho^(-2n) below 2^-52 (binary64, the
    // unit roundoff: even a cancellation of 1e4 in the sums leaves ~2e-12)
    // and 2^-26 (binary32)
    const double K64 = kRuleK64, K32 = kRuleK32;
    for (int n : ns) {
        if (n > kmax) break;
        std::vector<double> d, gam;
        if (!gauss_from_jacobi(n, alpha, beta, mu0, d, gam)) break;
        // moment check: exact for t^m, m < 2n
        bool ok = true;
        for (int m = 0; m < 2 * n && ok; ++m) {
            double a = 0.0, b = 0.0, sabs = 0.0;
            for (int j = 0; j < N; ++j) {
                double tm = std::pow(T.t[j], m);
                a += T.e[j] * tm;
                sabs += T.e[j] * tm;
            }
            for (int k = 0; k < n; ++k) b += gam[k] * std::pow(d[k], m);
            ok = std::fabs(a - b) <= 1e-11 * sabs;
        }
        if (!ok) break;
        int r = T.nrule++;
        T.rule_n[r] = n;
        T.rule_off[r] = T.rules_total;
        T.rho_min64[r] = (float)std::exp(K64 / n);
        T.rho_min32[r] = (float)std::exp(K32 / n);
        for (int k = 0; k < n; ++k) {
            r64.push_back(d[k]);
            r64.push_back(gam[k]);
            r64.push_back(gam[k] * d[k]);
            r32.push_back(make_float4((float)d[k], (float)gam[k], (float)(gam[k] * d[k]), 0.f));
        }
        T.rules_total += n;
    }
}

// Per (device, stream) scratch: calls on one stream are ordered by the
// stream, so they can share it; calls on different streams get their own.
// counters: [0] work counter of the first launch, [1] of the node-group
// launch and [9] of the binary64 list launch (mixed precision), [2] length of
// the binary64 list and [10] of the node list, [3] node evaluations, [4]
// angular pairs and [7] full-table pairs of the first launch, [6], [5] and
// [8] the same of the node-group launch, [12], [11] and [13] of the binary64
// list launch; the G0(mu2) kernel of every call zeroes them.
struct Scratch {
    double *partials = nullptr;   // 2 * kMaxG0Warps
    unsigned *ticket = nullptr;
    double *g0mu = nullptr;       // 2
    unsigned long long *counters = nullptr;   // kCounters
    int64_t *list = nullptr;      // binary64 list of the mixed precision
    int64_t list_cap = 0;
    NodeEntry *node_list = nullptr;   // partially routed points of the mixed precision
    int64_t node_list_cap = 0;
    float4 *snap = nullptr;       // the binary32 bulk's group snapshots
    int64_t snap_slots = 0;
    double *stage_x = nullptr, *stage_G = nullptr;   // host-path staging
    int64_t stage_cap = 0;
};

// what gfc_last_stats needs to read the counts of the last call
struct LastCall {
    unsigned long long *counters = nullptr;
    cudaStream_t stream = nullptr;
    int precision = GFC_FP64;
};
static thread_local LastCall g_last_call;

constexpr int kMaxG0Warps = 512;

struct DeviceState {
    std::map<std::tuple<int, int, int, double, int>, std::unique_ptr<Tables>> tables;
    std::map<cudaStream_t, std::unique_ptr<Scratch>> scratch;
};

static std::mutex g_mu;
static std::map<int, DeviceState> g_dev;

static int free_tables(Tables &T)
{
    cudaFree(T.rad64);
    cudaFree(T.rayp64);
    cudaFree(T.rayq_df);
    cudaFree(T.seg64);
    cudaFree(T.arc64);
    cudaFree(T.rad32);
    cudaFree(T.seg32);
    cudaFree(T.arc32);
    cudaFree(T.ang64);
    cudaFree(T.ang32);
    cudaFree(T.rules64);
    cudaFree(T.rules32);
    cudaFree(T.rad_df);
    cudaFree(T.tail64);
    cudaFree(T.tail32);
    cudaFree(T.tail_df);
    cudaFree(T.seg_df);
    cudaFree(T.arc_df);
    cudaFree(T.ang_df);
    cudaFree(T.rules_df);
    return GFC_OK;
}

template <typename V>
static int upload(V **dst, const std::vector<V> &src, size_t &bytes)
{
    size_t nb = sizeof(V) * src.size();
    cudaError_t e = dev_malloc((void **)dst, nb ? nb : sizeof(V));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(node table)");
    if (nb) {
        e = cudaMemcpy(*dst, src.data(), nb, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(node table)");
    }
    bytes += nb;
    return GFC_OK;
}

// Nodes z_j = cos psi_j (descending in z) and weights w_j of the angular rule
// for int_0^pi f(cos psi) sin^(D-2) psi dpsi (Sect. 4: tanh-sinh in z, with
// Gauss-Chebyshev rules of both kinds as a check; Gauss-Legendre in psi by
// default). Every rule is symmetric: z_(n-1-j) = -z_j.
static void angular_nodes(int rule, int n, int dim, std::vector<double> &z, std::vector<double> &w)
{
    const double pi = 3.14159265358979323846;
    auto sinpow = [dim](double s) { return dim == 4 ? s * s : s; };
    if (rule == GFC_ANG_TANH_SINH) {
        // trapezoid in s = k h on [-3, 3] for z = tanh(pi/2 sinh s); the
        // factor (1 - z^2)^(1/2) of D = 4 is 1/cosh(pi/2 sinh s) exactly
        const int N = (n - 1) / 2;
        const double h = 3.0 / N;
        for (int i = 0; i < n; ++i) {
            const double s = (N - i) * h, u = 0.5 * pi * std::sinh(s), cu = std::cosh(u);
            const double dz = h * 0.5 * pi * std::cosh(s) / (cu * cu);
            z[i] = std::tanh(u);
            w[i] = dim == 4 ? dz / cu : dz;
        }
        return;
    }
    if (rule == GFC_ANG_CHEBYSHEV1 || rule == GFC_ANG_CHEBYSHEV2) {
        const bool first = rule == GFC_ANG_CHEBYSHEV1;
        for (int i = 0; i < n; ++i) {
            const double psi = first ? (i + 0.5) * pi / n : (i + 1) * pi / (n + 1);
            z[i] = std::cos(psi);
            w[i] = (first ? pi / n : pi / (n + 1)) * sinpow(std::sin(psi));
        }
        return;
    }
    std::vector<double> gx, gw;
    gauss_legendre(n, gx, gw);
    for (int i = 0; i < n; ++i) {
        const double psi = 0.5 * pi * (gx[i] + 1.0);
        z[i] = std::cos(psi);
        w[i] = 0.5 * pi * gw[i] * sinpow(std::sin(psi));
    }
}

// The angular pair table (t_j = cos^2 psi_j, e_j = w_j t_j^2, g_j = e_j t_j)
// of T's angular rule, its moments Omega, Omega1 and delta, and its compressed
// rules (host only: the device copies are made by build_tables).
static void angular_host(Tables &T, std::vector<double> &ang64, std::vector<float> &ang32,
                         std::vector<double> &r64, std::vector<float4> &r32)
{
    // angular pairs: psi_j and pi - psi_j on [0, pi], weight w sin^(D-2) psi;
    // an odd rule's centre node psi = pi/2 pairs with itself at half weight
    // (none when the angular integral is taken in closed form)
    const bool exact = T.ang_rule == GFC_ANG_EXACT;
    std::vector<double> az(exact ? 0 : T.n_a), aw(exact ? 0 : T.n_a);
    if (!exact) angular_nodes(T.ang_rule, T.n_a, T.dim, az, aw);
    int np = exact ? 0 : (T.n_a + 1) / 2;
    T.t.resize(np);
    T.e.resize(np);
    T.g.resize(np);
    ang64.assign(3 * np, 0.0);
    ang32.assign(3 * np, 0.0f);
    double Om = 0, Om1 = 0, c_om = 0, c_om1 = 0;
    for (int j = 0; j < np; ++j) {
        const bool centre = 2 * j + 1 == T.n_a;
        double w = centre ? 0.5 * aw[j] : aw[j];
        double t = centre ? 0.0 : az[j] * az[j];
        T.t[j] = t;
        T.e[j] = w * t * t;
        T.g[j] = w * t * t * t;
        ang64[3 * j] = T.t[j];
        ang64[3 * j + 1] = T.e[j];
        ang64[3 * j + 2] = T.g[j];
        ang32[3 * j] = (float)T.t[j];
        ang32[3 * j + 1] = (float)T.e[j];
        ang32[3 * j + 2] = (float)T.g[j];
        // Kahan sums of the pair moments
        double y = w - c_om, s = Om + y;
        c_om = (s - Om) - y;
        Om = s;
        y = w * t - c_om1;
        s = Om1 + y;
        c_om1 = (s - Om1) - y;
        Om1 = s;
    }
    T.Omega = Om;
    T.Omega1 = Om1;
    T.delta = 4.0 * Om1 - Om;
    r64.clear();
    r32.clear();
    build_rules(T, r64, r32);
}

static int build_tables(Tables &T)
{
    const double pi = 3.14159265358979323846;
    std::vector<double> gx, gw;
    // radial: t = (1 + xi)/2 on (0, 1), |q| = L t/(1 - t), W = L/(1 - t)^2 w/2
    gauss_legendre(T.n_r, gx, gw);
    std::vector<double2> rad64(T.n_r), rayp64(T.n_r);
    std::vector<float2> rad32(T.n_r);
    for (int k = 0; k < T.n_r; ++k) {
        // 1 - t = (1 - xi)/2 computed without cancellation from the angle form
        double t = 0.5 * (gx[k] + 1.0), omt = 0.5 * (1.0 - gx[k]);
        double rho = T.L * t / omt, W = T.L / (omt * omt) * 0.5 * gw[k];
        rad64[k] = make_double2(rho, W);
        rad32[k] = make_float2((float)rho, (float)W);
        // the binary64 ray node's rho^2 and measure rho^(D-1) W, rounded as
        // the kernels would round them
        const double r2 = rho * rho;
        rayp64[k] = make_double2(r2, (T.dim == 4 ? r2 * rho : r2) * W);
    }
    // the clustered rule's tail: n_r/2 GL nodes on the same mapped half-line
    gauss_legendre(T.n_r / 2, gx, gw);
    std::vector<double2> tail64(T.n_r / 2);
    std::vector<float2> tail32(T.n_r / 2);
    for (int k = 0; k < T.n_r / 2; ++k) {
        double t = 0.5 * (gx[k] + 1.0), omt = 0.5 * (1.0 - gx[k]);
        double rho = T.L * t / omt, W = T.L / (omt * omt) * 0.5 * gw[k];
        tail64[k] = make_double2(rho, W);
        tail32[k] = make_float2((float)rho, (float)W);
    }
    // detour segments: n_r/4 GL nodes on [0, 1], and cos/sin(pi t) for arcs
    int ns = T.n_r / 4;
    gauss_legendre(ns, gx, gw);
    std::vector<double2> seg64(ns), arc64(ns);
    std::vector<float2> seg32(ns), arc32(ns);
    for (int k = 0; k < ns; ++k) {
        double t = 0.5 * (gx[k] + 1.0), w = 0.5 * gw[k];
        seg64[k] = make_double2(t, w);
        seg32[k] = make_float2((float)t, (float)w);
        arc64[k] = make_double2(std::cos(pi * t), std::sin(pi * t));
        arc32[k] = make_float2((float)std::cos(pi * t), (float)std::sin(pi * t));
    }
    std::vector<double> ang64, r64;
    std::vector<float> ang32;
    std::vector<float4> r32;
    angular_host(T, ang64, ang32, r64, r32);
    const int np = (int)T.t.size();
    // double-float copies (hi = nearest binary32, lo = the rest)
    auto dfv = [](double a) { df v(a); return make_float2(v.hi, v.lo); };
    auto df4 = [](double a, double b) {
        df u(a), v(b);
        return make_float4(u.hi, u.lo, v.hi, v.lo);
    };
    std::vector<float4> radD(T.n_r), segD(ns), arcD(ns), tailD(T.n_r / 2);
    for (int k = 0; k < T.n_r; ++k) radD[k] = df4(rad64[k].x, rad64[k].y);
    // the double-float ray nodes in the frame of the ray, scaled by
    // s = 1/(1 + rho^2) so that every node quantity stays within binary32's
    // range (rho^2 reaches ~1e12 at 2048 nodes)
    std::vector<float4> rayqD(2 * T.n_r);
    for (int k = 0; k < T.n_r; ++k) {
        const double r2 = rayp64[k].x, s = 1.0 / (1.0 + r2);
        rayqD[2 * k] = df4(r2 * s, s);
        rayqD[2 * k + 1] = df4(rayp64[k].y * s * s * s, 0.0);
    }
    for (int k = 0; k < T.n_r / 2; ++k) tailD[k] = df4(tail64[k].x, tail64[k].y);
    for (int k = 0; k < ns; ++k) {
        segD[k] = df4(seg64[k].x, seg64[k].y);
        arcD[k] = df4(arc64[k].x, arc64[k].y);
    }
    std::vector<float2> angD(3 * np), rulesD(r64.size());
    for (int j = 0; j < 3 * np; ++j) angD[j] = dfv(ang64[j]);
    for (size_t j = 0; j < r64.size(); ++j) rulesD[j] = dfv(r64[j]);
    int st;
    if ((st = upload(&T.rad64, rad64, T.bytes)) || (st = upload(&T.rad32, rad32, T.bytes)) ||
        (st = upload(&T.rayp64, rayp64, T.bytes)) || (st = upload(&T.rayq_df, rayqD, T.bytes)) ||
        (st = upload(&T.seg64, seg64, T.bytes)) || (st = upload(&T.seg32, seg32, T.bytes)) ||
        (st = upload(&T.arc64, arc64, T.bytes)) || (st = upload(&T.arc32, arc32, T.bytes)) ||
        (st = upload(&T.ang64, ang64, T.bytes)) || (st = upload(&T.ang32, ang32, T.bytes)) ||
        (st = upload(&T.rules64, r64, T.bytes)) || (st = upload(&T.rules32, r32, T.bytes)) ||
        (st = upload(&T.rad_df, radD, T.bytes)) || (st = upload(&T.seg_df, segD, T.bytes)) ||
        (st = upload(&T.arc_df, arcD, T.bytes)) || (st = upload(&T.ang_df, angD, T.bytes)) ||
        (st = upload(&T.rules_df, rulesD, T.bytes)) || (st = upload(&T.tail64, tail64, T.bytes)) ||
        (st = upload(&T.tail32, tail32, T.bytes)) || (st = upload(&T.tail_df, tailD, T.bytes)))
        return st;
    return GFC_OK;
}

static int get_device(int *dev)
{
    cudaError_t e = cudaGetDevice(dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    return GFC_OK;
}

int get_tables(int dev, int n_r, int n_a, int dim, double L, int ang_rule, Tables **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto &ds = g_dev[dev];
    auto key = std::make_tuple(n_r, n_a, dim, L, ang_rule);
    auto it = ds.tables.find(key);
    if (it != ds.tables.end()) {
        *out = it->second.get();
        return GFC_OK;
    }
    auto T = std::make_unique<Tables>();
    T->n_r = n_r;
    T->n_a = n_a;
    T->dim = dim;
    T->L = L;
    T->ang_rule = ang_rule;
    int st = build_tables(*T);
    if (st != GFC_OK) {
        free_tables(*T);
        return st;
    }
    *out = T.get();
    ds.tables[key] = std::move(T);
    return GFC_OK;
}

int get_scratch(int dev, cudaStream_t s, Scratch **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto &ds = g_dev[dev];
    auto it = ds.scratch.find(s);
    if (it != ds.scratch.end()) {
        *out = it->second.get();
        return GFC_OK;
    }
    auto S = std::make_unique<Scratch>();
    cudaError_t e;
    if ((e = dev_malloc((void **)&S->partials, sizeof(double) * 2 * kMaxG0Warps)) != cudaSuccess ||
        (e = dev_malloc((void **)&S->ticket, sizeof(unsigned))) != cudaSuccess ||
        (e = dev_malloc((void **)&S->g0mu, sizeof(double) * 2)) != cudaSuccess ||
        (e = dev_malloc((void **)&S->counters, sizeof(unsigned long long) * kCounters)) != cudaSuccess) {
        cudaFree(S->partials);
        cudaFree(S->ticket);
        cudaFree(S->g0mu);
        cudaFree(S->counters);
        return cuda_fail(e, "cudaMalloc(scratch)");
    }
    e = cudaMemset(S->ticket, 0, sizeof(unsigned));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(scratch)");
    *out = S.get();
    ds.scratch[s] = std::move(S);
    return GFC_OK;
}

// ---------------------------------------------------------------------------
// argument checks and per-propagator constants
// ---------------------------------------------------------------------------
static int check_params(const gfc_params *p)
{
    if (!p) return fail(GFC_EINVAL, "params is NULL");
    if (p->dim != 3 && p->dim != 4) return fail(GFC_EINVAL, "dim must be 3 or 4");
    if (!(p->mu2 >= 0.0) || !std::isfinite(p->mu2)) return fail(GFC_EINVAL, "mu2 must be >= 0");
    if (p->n_radial < 4 || p->n_radial > kMaxRadial || p->n_radial % 4)
        return fail(GFC_EINVAL, "n_radial must be a multiple of 4 in [4, 16384]");
    if (p->n_angular < 2 || p->n_angular > kMaxAngular)
        return fail(GFC_EINVAL, "n_angular must be in [2, 512]");
    if (p->angular_rule < GFC_ANG_GAUSS_LEGENDRE || p->angular_rule > GFC_ANG_EXACT)
        return fail(GFC_EINVAL, "angular_rule must be a gfc_angular_rule");
    if (p->radial_rule != GFC_RAD_MAPPED && p->radial_rule != GFC_RAD_CLUSTERED)
        return fail(GFC_EINVAL, "radial_rule must be a gfc_radial_rule");
    if (p->angular_rule == GFC_ANG_TANH_SINH && (p->n_angular % 2 == 0 || p->n_angular < 3))
        return fail(GFC_EINVAL, "the tanh-sinh rule needs an odd n_angular >= 3");
    if (!(p->radial_scale > 0.0) || !std::isfinite(p->radial_scale))
        return fail(GFC_EINVAL, "radial_scale must be > 0");
    if (!(p->detour_radius > 0.0)) return fail(GFC_EINVAL, "detour_radius must be > 0");
    if (p->precision != GFC_FP64 && p->precision != GFC_MIXED && p->precision != GFC_F32X2)
        return fail(GFC_EINVAL, "precision must be GFC_FP64, GFC_MIXED or GFC_F32X2");
    if (p->mixed_fallback != GFC_FP64 && p->mixed_fallback != GFC_F32X2)
        return fail(GFC_EINVAL, "mixed_fallback must be GFC_FP64 or GFC_F32X2");
    if (!(p->cut_band >= 0.0) || !(p->pinch_angle >= 0.0) || !(p->mixed_rtol >= 0.0))
        return fail(GFC_EINVAL, "cut_band, pinch_angle and mixed_rtol must be >= 0");
    return GFC_OK;
}

int make_prop(const gfc_propagator *g, const gfc_params *p, PropConst &pc)
{
    if (!g) return fail(GFC_EINVAL, "propagator is NULL");
    std::memset(&pc, 0, sizeof pc);
    pc.kind = g->kind;
    pc.pinch = -1.0;
    const double pi = 3.14159265358979323846;
    if (g->kind == GFC_PROP_SCALAR) {
        if (!(g->m2 > 0.0) || !std::isfinite(g->m2)) return fail(GFC_EINVAL, "SCALAR needs m2 > 0");
        pc.m2 = g->m2;
        pc.thr = -4.0 * g->m2;
        pc.pinch = pi;
    } else if (g->kind == GFC_PROP_CPAIR) {
        if (g->mk2_re != g->mq2_re || g->mk2_im != -g->mq2_im || g->mk2_im == 0.0)
            return fail(GFC_EINVAL, "CPAIR needs Mq2 = conj(Mk2) with Im Mk2 != 0");
        std::complex<double> Mk(g->mk2_re, g->mk2_im), Mq(g->mq2_re, g->mq2_im);
        std::complex<double> yk0 = -Mk, yq0 = -Mq;
        std::complex<double> yu = yk0.imag() > 0 ? yk0 : yq0;
        pc.yu_re = yu.real();
        pc.yu_im = yu.imag();
        pc.arg_yu = std::arg(yu);
        pc.yk0_re = yk0.real();
        pc.yk0_im = yk0.imag();
        if (!(p->detour_radius < 0.5 * std::abs(yu)))
            return fail(GFC_EINVAL, "detour_radius must be below half the pole modulus");
        std::complex<double> S = std::sqrt(Mk) + std::sqrt(Mq);
        pc.thr = -(S * S).real();
    } else if (g->kind == GFC_PROP_DRESSED) {
        double a = g->a, b = g->b, c = g->c;
        if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c) || !(4 * c - b * b > 0.0))
            return fail(GFC_EINVAL, "DRESSED needs b^2 < 4c (complex-conjugate poles)");
        std::complex<double> yp(-0.5 * b, 0.5 * std::sqrt(4 * c - b * b)), ym = std::conj(yp);
        std::complex<double> Rp = (yp + a) / (yp - ym);
        pc.a = a;
        pc.b = b;
        pc.c = c;
        pc.yp_re = yp.real();
        pc.yp_im = yp.imag();
        pc.Rp_re = Rp.real();
        pc.Rp_im = Rp.imag();
        pc.arg_yp = std::arg(yp);
        if (!(p->detour_radius < 0.5 * std::abs(yp)))
            return fail(GFC_EINVAL, "detour_radius must be below half the pole modulus");
        std::complex<double> S = std::sqrt(-yp) + std::sqrt(-ym);
        pc.thr = -(S * S).real();
        pc.pinch = pc.arg_yp;
    } else {
        return fail(GFC_EINVAL, "unknown propagator kind");
    }
    return GFC_OK;
}

static void fill_kparams_tables(KParams &kp, const gfc_params *p, const Tables &T,
                                const PropConst &pc)
{
    std::memset(&kp, 0, sizeof kp);
    const double pi = 3.14159265358979323846;
    kp.dim = p->dim;
    kp.n_r = p->n_radial;
    kp.n_s = p->n_radial / 4;
    kp.npair = npair_of(p);
    kp.ang_exact = p->angular_rule == GFC_ANG_EXACT;
    kp.rad64 = T.rad64;
    kp.rayp64 = T.rayp64;
    kp.rayq_df = T.rayq_df;
    kp.rad32 = T.rad32;
    kp.seg64 = T.seg64;
    kp.seg32 = T.seg32;
    kp.arc64 = T.arc64;
    kp.arc32 = T.arc32;
    kp.rad_df = T.rad_df;
    kp.tail64 = T.tail64;
    kp.tail32 = T.tail32;
    kp.tail_df = T.tail_df;
    kp.radial_rule = p->radial_rule;
    kp.seg_df = T.seg_df;
    kp.arc_df = T.arc_df;
    kp.rules_df = T.rules_df;
    kp.L = p->radial_scale;
    kp.r_detour = p->detour_radius;
    // K_D = S_(D-2)/(2 pi)^D, eq. 11 for D = 4
    kp.K_D = p->dim == 4 ? 4.0 * pi / std::pow(2.0 * pi, 4) : 2.0 * pi / std::pow(2.0 * pi, 3);
    kp.Omega = T.Omega;
    kp.Omega1 = T.Omega1;
    kp.delta = T.delta;
    kp.nrule = full_rule_forced() ? 0 : T.nrule;
    for (int r = 0; r < T.nrule; ++r) {
        kp.rule_off[r] = T.rule_off[r];
        kp.rule_n[r] = T.rule_n[r];
        kp.sig_min32[r] = (float)(0.5 * ((double)T.rho_min32[r] + 1.0 / (double)T.rho_min32[r]));
        kp.sig_min64[r] = (float)(0.5 * ((double)T.rho_min64[r] + 1.0 / (double)T.rho_min64[r]));
    }
    // the selection as an index: rho_min[r] = exp(K / rule_n[r]) (build_rules)
    kp.rule_k32 = (float)kRuleK32;
    kp.rule_k64 = (float)kRuleK64;
    for (int m = 0; m < 128; ++m) {
        int r = 0;
        while (r < kp.nrule && kp.rule_n[r] < m) ++r;
        kp.rule_idx[m] = (unsigned char)r;
    }
    kp.rules64 = T.rules64;
    kp.rules32 = T.rules32;
    kp.rules_total = T.rules_total;
    kp.pc = pc;
    {
        const double c[6] = {kp.Omega1, kp.delta, pc.yp_re, pc.yp_im, pc.Rp_re, pc.Rp_im};
        for (int i = 0; i < 6; ++i) {
            df v(c[i]);
            kp.f32c[i] = (float)c[i];
            kp.dfc[2 * i] = v.hi;
            kp.dfc[2 * i + 1] = v.lo;
        }
        const df om(kp.Omega);
        kp.om_df[0] = om.hi;
        kp.om_df[1] = om.lo;
    }
    kp.cut_band = p->cut_band;
    kp.pinch_angle = p->pinch_angle;
    kp.mixed_rtol = p->mixed_rtol;
    kp.mu2 = p->mu2;
}

static void fill_kparams(KParams &kp, const gfc_params *p, const Tables &T, const PropConst &pc,
                         Scratch &S)
{
    fill_kparams_tables(kp, p, T, pc);
    kp.g0mu = S.g0mu;
    kp.counter = S.counters;
    kp.list = S.list;
    kp.list_count = S.counters + 2;
    kp.node_count = S.counters + 3;
    kp.pair_count = S.counters + 4;
    kp.pair_full_count = S.counters + 7;
}

static int grow_list(Scratch &S, int64_t n)
{
    if (S.list_cap >= n) return GFC_OK;
    cudaFree(S.list);
    S.list = nullptr;
    S.list_cap = 0;
    cudaError_t e = dev_malloc((void **)&S.list, sizeof(int64_t) * (n > 0 ? n : 1));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(binary64 list)");
    S.list_cap = n;
    return GFC_OK;
}

// The node list (one entry per point at most) and the bulk's snapshots: one
// slot of kMaxGroups x 32 float4 per warp the binary32 bulk can have resident
// (every SM at 8 blocks of 256 threads, the most 2048 threads allow).
static int grow_partial(Scratch &S, int64_t n)
{
    if (S.node_list_cap < n) {
        cudaFree(S.node_list);
        S.node_list = nullptr;
        S.node_list_cap = 0;
        cudaError_t e = dev_malloc((void **)&S.node_list, sizeof(NodeEntry) * (n > 0 ? n : 1));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(node list)");
        S.node_list_cap = n;
    }
    if (!S.snap) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const int64_t slots = (int64_t)(sms > 0 ? sms : 1) * 8 * 8;
        cudaError_t e = dev_malloc((void **)&S.snap, sizeof(float4) * kMaxGroups * 32 * slots);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(group snapshots)");
        S.snap_slots = slots;
    }
    return GFC_OK;
}

static DevTables dev_tables(const Tables &T)
{
    DevTables tb;
    tb.ang64 = T.ang64;
    tb.ang32 = T.ang32;
    tb.ang_df = T.ang_df;
    tb.t = T.t.data();
    tb.e = T.e.data();
    tb.g = T.g.data();
    return tb;
}

// One evaluation on `st`: G0(mu2) (which also resets the work counters),
// then the points, in one or two launches.
static int run(const gfc_propagator *prop, const gfc_params *p, KParams kp_points,
               cudaStream_t st, double *cond_out)
{
    NvtxRange nvtx("gfc_eval");
    PropConst pc;
    int rc = make_prop(prop, p, pc);
    if (rc) return rc;
    int dev;
    if ((rc = get_device(&dev))) return rc;
    Tables *T;
    if ((rc = get_tables(dev, p->n_radial, p->n_angular, p->dim, p->radial_scale, p->angular_rule,
                         &T)))
        return rc;
    Scratch *S;
    if ((rc = get_scratch(dev, st, &S))) return rc;
    if (p->precision == GFC_MIXED &&
        ((rc = grow_list(*S, kp_points.npts)) || (rc = grow_partial(*S, kp_points.npts))))
        return rc;
    KParams kp;
    fill_kparams(kp, p, *T, pc, *S);
    kp.cond_out = cond_out;
    kp.use_grid = kp_points.use_grid;
    kp.npts = kp_points.npts;
    kp.re0 = kp_points.re0;
    kp.dre = kp_points.dre;
    kp.im0 = kp_points.im0;
    kp.dim_im = kp_points.dim_im;
    kp.gm = kp_points.gm;
    kp.gn = kp_points.gn;
    kp.x = kp_points.x;
    kp.G = kp_points.G;
    DevTables tb = dev_tables(*T);
    gfc_eval_stats stats{};
    stats.points = kp.npts;
    int nw = (p->n_radial + 31) / 32;
    if (nw > kMaxG0Warps) nw = kMaxG0Warps;
    cudaError_t e = launch_g0mu(kp, tb, p->mu2, S->partials, nw, S->ticket, S->g0mu, S->counters,
                                st);
    if (e != cudaSuccess) return cuda_fail(e, "g0mu launch");
    stats.kernel_launches = 1;
    if (kp.npts > 0) {
        if (p->precision != GFC_MIXED) {
            kp.mode = MODE_ALL;
            kp.counter = S->counters;
            e = launch_eval(kp, tb, p->precision == GFC_F32X2 ? ARITH_DF : ARITH_F64, st);
            if (e != cudaSuccess) return cuda_fail(e, "eval launch");
            stats.kernel_launches += 1;
        } else {
            // the binary32 bulk; points it routes go whole (cut band, pinch)
            // to the binary64 list or with their worst node groups to the
            // node list
            kp.mode = MODE_BULK32;
            kp.counter = S->counters;
            kp.node_list = S->node_list;
            kp.node_list_count = S->counters + 10;
            kp.snap = S->snap;
            kp.snap_slots = S->snap_slots;
            e = launch_eval(kp, tb, ARITH_F32, st);
            if (e != cudaSuccess) return cuda_fail(e, "eval launch (binary32)");
            // the node groups in the fallback arithmetic, counted apart
            kp.mode = MODE_NODES;
            kp.counter = S->counters + 1;
            kp.pair_count = S->counters + 5;
            kp.node_count = S->counters + 6;
            kp.pair_full_count = S->counters + 8;
            e = launch_eval(kp, tb, p->mixed_fallback == GFC_F32X2 ? ARITH_DF : ARITH_F64, st);
            if (e != cudaSuccess) return cuda_fail(e, "eval launch (node groups)");
            // the whole points in binary64
            kp.mode = MODE_LIST64;
            kp.counter = S->counters + 9;
            kp.pair_count = S->counters + 11;
            kp.node_count = S->counters + 12;
            kp.pair_full_count = S->counters + 13;
            e = launch_eval(kp, tb, ARITH_F64, st);
            if (e != cudaSuccess) return cuda_fail(e, "eval launch (binary64 list)");
            stats.kernel_launches += 3;
        }
    }
    stats.points_fp64 = p->precision != GFC_MIXED ? kp.npts : -1;
    stats.node_evals = -1;
    g_last_stats = stats;
    g_last_call.counters = S->counters;
    g_last_call.stream = st;
    g_last_call.precision = p->precision;
    return GFC_OK;
}

// entry points for the serving runtime (void* keeps gfc.h out of the
// kernel-side header)
int check_params_c(const void *params) { return check_params((const gfc_params *)params); }

int make_prop_c(const void *prop, const void *params, PropConst &pc)
{
    return make_prop((const gfc_propagator *)prop, (const gfc_params *)params, pc);
}

int get_tables_c(int dev, int n_r, int n_a, int dim, double L, int ang_rule, Tables **out,
                 size_t *bytes)
{
    int rc = get_tables(dev, n_r, n_a, dim, L, ang_rule, out);
    if (rc == GFC_OK && bytes) *bytes = (*out)->bytes;
    return rc;
}

void fill_kparams_c(KParams &kp, const void *params, const Tables &T, const PropConst &pc)
{
    fill_kparams_tables(kp, (const gfc_params *)params, T, pc);
}

DevTables dev_tables_c(const Tables &T) { return dev_tables(T); }

}  // namespace gfc

using namespace gfc;

extern "C" {

const char *gfc_strerror(int status)
{
    switch (status) {
    case GFC_OK: return "ok";
    case GFC_EINVAL: return "invalid argument";
    case GFC_ENOMEM: return "out of memory";
    case GFC_EBUDGET: return "request exceeds the memory budget";
    case GFC_ECUDA: return "CUDA runtime error";
    case GFC_ETIMEOUT: return "timed out";
    case GFC_ECANCELED: return "cancelled";
    case GFC_EBUSY: return "busy";
    case GFC_ENOTFOUND: return "unknown ticket";
    default: return "unknown status";
    }
}

const char *gfc_last_error(void) { return g_last_error.c_str(); }

int gfc_version(int *major, int *minor)
{
    if (major) *major = GFC_VERSION_MAJOR;
    if (minor) *minor = GFC_VERSION_MINOR;
    return GFC_OK;
}

int gfc_params_default(gfc_params *p)
{
    if (!p) return fail(GFC_EINVAL, "params is NULL");
    std::memset(p, 0, sizeof *p);
    p->dim = 4;
    p->mu2 = 1.0;
    p->n_radial = 2048;
    p->n_angular = 256;
    p->radial_scale = 1.0;
    p->detour_radius = 0.1;
    p->precision = GFC_FP64;
    p->cut_band = 0.05;
    p->pinch_angle = 0.0;
    p->mixed_rtol = 1e-6;
    p->mixed_fallback = GFC_F32X2;
    p->angular_rule = GFC_ANG_GAUSS_LEGENDRE;
    p->radial_rule = GFC_RAD_MAPPED;
    return GFC_OK;
}

int gfc_eval_points(const gfc_propagator *prop, const gfc_params *params, const double *x,
                    int64_t npts, double *G, void *stream)
{
    g_last_error.clear();
    int rc = check_params(params);
    if (rc) return rc;
    if (npts < 0) return fail(GFC_EINVAL, "npts < 0");
    if (npts > 0 && (!x || !G)) return fail(GFC_EINVAL, "x and G must be device pointers");
    if (((uintptr_t)x | (uintptr_t)G) & 15) return fail(GFC_EINVAL, "x and G must be 16-byte aligned");
    KParams kp{};
    kp.use_grid = 0;
    kp.npts = npts;
    kp.x = x;
    kp.G = G;
    return run(prop, params, kp, (cudaStream_t)stream, nullptr);
}

int gfc_eval_points_cond(const gfc_propagator *prop, const gfc_params *params, const double *x,
                         int64_t npts, double *G, double *cond, void *stream)
{
    g_last_error.clear();
    int rc = check_params(params);
    if (rc) return rc;
    if (npts < 0) return fail(GFC_EINVAL, "npts < 0");
    if (npts > 0 && (!x || !G)) return fail(GFC_EINVAL, "x and G must be device pointers");
    if (((uintptr_t)x | (uintptr_t)G) & 15) return fail(GFC_EINVAL, "x and G must be 16-byte aligned");
    if (((uintptr_t)cond) & 7) return fail(GFC_EINVAL, "cond must be 8-byte aligned");
    KParams kp{};
    kp.use_grid = 0;
    kp.npts = npts;
    kp.x = x;
    kp.G = G;
    return run(prop, params, kp, (cudaStream_t)stream, cond);
}

static int check_grid(const gfc_grid *g)
{
    if (!g) return fail(GFC_EINVAL, "grid is NULL");
    if (g->m < 1 || g->n < 1) return fail(GFC_EINVAL, "grid needs m, n >= 1");
    if ((int64_t)g->m * g->n > (int64_t)1 << 34) return fail(GFC_EINVAL, "grid too large");
    if (!std::isfinite(g->re0) || !std::isfinite(g->re1) || !std::isfinite(g->im0) ||
        !std::isfinite(g->im1) || !(g->re1 > g->re0) || !(g->im1 > g->im0))
        return fail(GFC_EINVAL, "grid needs re0 < re1 and im0 < im1");
    return GFC_OK;
}

}  // extern "C"

int gfc::check_grid_c(const void *grid)
{
    const gfc_grid *g = (const gfc_grid *)grid;
    int rc = check_grid(g);
    if (rc) return rc;
    double dre = (g->re1 - g->re0) / g->m, dim = (g->im1 - g->im0) / g->n;
    for (int j = 0; j < g->n; ++j) {
        double xi = g->im0 + (j + 0.5) * dim;
        if (xi == 0.0 && g->re0 + 0.5 * dre < 0.0)
            return fail(GFC_EINVAL, "a grid row lies on the negative real axis");
    }
    return GFC_OK;
}

extern "C" {

int gfc_eval_grid(const gfc_propagator *prop, const gfc_params *params, const gfc_grid *grid,
                  double *G, void *stream)
{
    g_last_error.clear();
    int rc = check_params(params);
    if (rc) return rc;
    if ((rc = check_grid(grid))) return rc;
    if (!G || ((uintptr_t)G & 15)) return fail(GFC_EINVAL, "G must be a 16-byte aligned device pointer");
    double dre = (grid->re1 - grid->re0) / grid->m, dim = (grid->im1 - grid->im0) / grid->n;
    // a grid row on the real axis with Re x < 0 would sit on the cut side
    for (int j = 0; j < grid->n; ++j) {
        double xi = grid->im0 + (j + 0.5) * dim;
        if (xi == 0.0 && grid->re0 + 0.5 * dre < 0.0)
            return fail(GFC_EINVAL, "a grid row lies on the negative real axis");
    }
    KParams kp{};
    kp.use_grid = 1;
    kp.npts = (int64_t)grid->m * grid->n;
    kp.re0 = grid->re0;
    kp.dre = dre;
    kp.im0 = grid->im0;
    kp.dim_im = dim;
    kp.gm = grid->m;
    kp.gn = grid->n;
    kp.G = G;
    return run(prop, params, kp, (cudaStream_t)stream, nullptr);
}

int gfc_grid_points(const gfc_grid *grid, double *x, void *stream)
{
    g_last_error.clear();
    int rc = check_grid(grid);
    if (rc) return rc;
    if (!x || ((uintptr_t)x & 15)) return fail(GFC_EINVAL, "x must be a 16-byte aligned device pointer");
    double dre = (grid->re1 - grid->re0) / grid->m, dim = (grid->im1 - grid->im0) / grid->n;
    cudaError_t e = launch_grid_points(grid->re0, dre, grid->im0, dim, grid->m, grid->n, x,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "grid launch");
    return GFC_OK;
}

int gfc_eval_points_host(const gfc_propagator *prop, const gfc_params *params,
                         const double *x_host, int64_t npts, double *G_host, void *stream)
{
    g_last_error.clear();
    int rc = check_params(params);
    if (rc) return rc;
    if (npts < 0) return fail(GFC_EINVAL, "npts < 0");
    if (npts == 0) return GFC_OK;
    if (!x_host || !G_host) return fail(GFC_EINVAL, "x_host and G_host must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int dev;
    if ((rc = get_device(&dev))) return rc;
    Scratch *S;
    if ((rc = get_scratch(dev, st, &S))) return rc;
    if (S->stage_cap < npts) {
        cudaFree(S->stage_x);
        cudaFree(S->stage_G);
        S->stage_x = S->stage_G = nullptr;
        S->stage_cap = 0;
        cudaError_t e;
        if ((e = dev_malloc((void **)&S->stage_x, 16 * npts)) != cudaSuccess ||
            (e = dev_malloc((void **)&S->stage_G, 16 * npts)) != cudaSuccess)
            return cuda_fail(e, "cudaMalloc(staging)");
        S->stage_cap = npts;
    }
    cudaError_t e = cudaMemcpyAsync(S->stage_x, x_host, 16 * npts, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(H2D)");
    if ((rc = gfc_eval_points(prop, params, S->stage_x, npts, S->stage_G, stream))) return rc;
    e = cudaMemcpyAsync(G_host, S->stage_G, 16 * npts, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(D2H)");
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    return GFC_OK;
}

int gfc_last_stats(gfc_eval_stats *out)
{
    if (!out) return fail(GFC_EINVAL, "out is NULL");
    *out = g_last_stats;
    if (g_last_call.counters) {
        unsigned long long c[kCounters];
        cudaError_t e = cudaStreamSynchronize(g_last_call.stream);
        if (e == cudaSuccess)
            e = cudaMemcpy(c, g_last_call.counters, sizeof c, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "reading the call's counters");
        out->node_evals = (int64_t)(c[3] + c[6] + c[12]);
        out->pairs_evaluated = (int64_t)(c[4] + c[5] + c[11]);
        out->pairs_full_table = (int64_t)(c[7] + c[8] + c[13]);
        out->node_evals_fallback = (int64_t)c[6];
        out->pairs_fallback = (int64_t)c[5];
        out->pairs_full_table_fallback = (int64_t)c[8];
        out->node_evals_list64 = (int64_t)c[12];
        out->pairs_list64 = (int64_t)c[11];
        out->pairs_full_table_list64 = (int64_t)c[13];
        if (g_last_call.precision == GFC_MIXED) {
            out->points_fp64 = (int64_t)c[2];
            out->points_partial = (int64_t)c[10];
        }
    }
    return GFC_OK;
}

int gfc_release(void)
{
    int dev;
    int rc = get_device(&dev);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_dev.find(dev);
    if (it == g_dev.end()) return GFC_OK;
    for (auto &kv : it->second.tables) free_tables(*kv.second);
    for (auto &kv : it->second.scratch) {
        Scratch &S = *kv.second;
        cudaFree(S.partials);
        cudaFree(S.ticket);
        cudaFree(S.g0mu);
        cudaFree(S.counters);
        cudaFree(S.node_list);
        cudaFree(S.snap);
        cudaFree(S.list);
        cudaFree(S.stage_x);
        cudaFree(S.stage_G);
    }
    g_dev.erase(it);
    return GFC_OK;
}

}  // extern "C"

extern "C" int gfc_test_fail_allocations(int n)
{
    if (n < 0) return gfc::fail(GFC_EINVAL, "n must be >= 0");
    gfc::g_fail_allocs.store(n);
    return GFC_OK;
}

extern "C" int gfc_test_fail_launches(int n)
{
    if (n < 0) return gfc::fail(GFC_EINVAL, "n must be >= 0");
    gfc::g_fail_launches.store(n);
    return GFC_OK;
}

extern "C" int gfc_test_full_angular_rule(int on)
{
    gfc::g_full_rule.store(on ? 1 : 0);
    return GFC_OK;
}

extern "C" int gfc_test_angular_rules(int n_angular, int dim, int angular_rule, double *pairs,
                                      int max_pairs, int *npair, double *rules, int max_rule_nodes,
                                      int *rule_n, float *rho_min, int *nrule)
{
    using namespace gfc;
    if (!npair || !nrule) return fail(GFC_EINVAL, "npair and nrule must not be NULL");
    gfc_params p;
    gfc_params_default(&p);
    p.dim = dim;
    p.n_angular = n_angular;
    p.angular_rule = angular_rule;
    int rc = check_params(&p);
    if (rc) return rc;
    Tables T;
    T.n_r = p.n_radial;
    T.n_a = n_angular;
    T.dim = dim;
    T.ang_rule = angular_rule;
    T.L = p.radial_scale;
    std::vector<double> ang64, r64;
    std::vector<float> ang32;
    std::vector<float4> r32;
    angular_host(T, ang64, ang32, r64, r32);
    const int np = (int)T.t.size();
    if (pairs && np > max_pairs) return fail(GFC_EINVAL, "pairs: capacity below the pair count");
    if (rules && T.rules_total > max_rule_nodes)
        return fail(GFC_EINVAL, "rules: capacity below the rule node count");
    *npair = np;
    *nrule = T.nrule;
    if (pairs) std::copy(ang64.begin(), ang64.end(), pairs);
    if (rules) std::copy(r64.begin(), r64.end(), rules);
    for (int r = 0; r < T.nrule; ++r) {
        if (rule_n) rule_n[r] = T.rule_n[r];
        if (rho_min) rho_min[r] = T.rho_min64[r];
    }
    return GFC_OK;
}
