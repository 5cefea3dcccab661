// Device code of libgfc for sm_103a: Kernel 1 (grid, Step 4) fused into
// Kernel 2 (the 2-D quadrature per point, Step 5) of Sect. 4 of the paper.
// Included by gfc_kernels.cu (G0(mu2), grid points, dispatch) and by
// gfc_eval_inst.cu, which is compiled once per (arithmetic, angular pair
// count) so that the instantiations build in parallel.
//
// Work layout: one warp per point of x (dynamic assignment through an atomic
// counter); the 32 lanes split the radial nodes of the point's contour; each
// lane runs the whole angular sum of its node, over the smallest compressed
// Gauss rule of the angular measure that is exact to rounding for the node
// (shared memory, uniform over the warp) or over the full table, held in the
// kernel's constant bank and fully unrolled. The angular sum is paired
// (psi, pi - psi) and written in a
// square-root-free, leading-order-subtracted form:
//
//   sum_j w_j (v t_j - 1)/(1 - w t_j)
//     = (delta y - Omega (x + M2)) / a - Omega1 w + (v - w) w T2,
//   T2 = sum_j w_j t_j^2 / (1 - w t_j) = A - conj(w) B,
//   A = sum_j w_j t_j^2 / |1 - w t_j|^2,  B = sum_j w_j t_j^3 / |1 - w t_j|^2,
//
// with a = x + y + M2, v = 4y/a, w = 4xy/a^2, t_j = cos^2 psi_j, Omega =
// sum w_j, Omega1 = sum w_j t_j, delta = 4 Omega1 - Omega. This is the
// combined-fraction integrand of eq. 20 summed over the symmetric pair; each
// pair costs one real reciprocal and a handful of FMAs, and A, B are sums of
// positive terms. The radial sum is compensated (TwoSum) in the binary32 path,
// carried in double-float by the double-float kernels and summed plainly in
// binary64, whose rounding there lies far below the FP64 tolerance.
#pragma once

#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "gfc_df.h"
#include "gfc_internal.h"

namespace gfc {

// calibration of the binary32 error estimate (multiple of 2^-24 per unit of
// the nodes' error scale), from binary32-vs-FP64 runs over the test grids
constexpr double kMixedErrFactor = 2.0;
constexpr float kMixedPinchQ = 1e-5f;   // |1 - w t|^2 below which a point is routed
// partial routing: the kept node groups' error estimate must pass with this
// margin (the estimate's spread around the error is wider once the largest
// groups are gone)
#ifndef GFC_PARTIAL_MARGIN
#define GFC_PARTIAL_MARGIN 4.0
#endif
constexpr double kPartialMargin = GFC_PARTIAL_MARGIN;
// partial routing applies to points whose estimate fails by at most this
// factor; beyond it every group is evaluated again
#ifndef GFC_PARTIAL_MAX
#define GFC_PARTIAL_MAX 32.0
#endif
constexpr double kPartialMax = GFC_PARTIAL_MAX;
// weight of the pole terms of kappa on binary32 ray nodes with y exact
#ifndef GFC_POLE_WEIGHT
#define GFC_POLE_WEIGHT 0.5
#endif
constexpr double kMixedPoleWeight = GFC_POLE_WEIGHT;

// ----------------------------------------------------------------------------
// complex arithmetic
// ----------------------------------------------------------------------------
template <typename T>
struct C {
    T r, i;
};

template <typename T>
__device__ __forceinline__ C<T> cx(T r, T i) { return C<T>{r, i}; }
template <typename T>
__device__ __forceinline__ C<T> operator+(C<T> a, C<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T>
__device__ __forceinline__ C<T> operator-(C<T> a, C<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T>
__device__ __forceinline__ C<T> operator*(C<T> a, C<T> b)
{
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
// double-float: each component as one product and one fused a b + c
template <>
__device__ __forceinline__ C<df> operator*(C<df> a, C<df> b)
{
    return {fma(a.r, b.r, -(a.i * b.i)), fma(a.r, b.i, a.i * b.r)};
}
template <typename T>
__device__ __forceinline__ C<T> operator*(T s, C<T> a) { return {s * a.r, s * a.i}; }
template <typename T>
__device__ __forceinline__ C<T> conj(C<T> a) { return {a.r, -a.i}; }

__device__ __forceinline__ float rcp(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1/x in binary64: hardware seed, then one order-3 Newton-Raphson step,
// r <- r (1 + e + e^2) with e = 1 - x r (the truncated series of 1/(1 - e)),
// which takes a seed error e to e^3.
__device__ __forceinline__ double rcp(double x)
{
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    return fma(r, fma(e, e, e), r);
}

template <typename T>
__device__ __forceinline__ C<T> cinv(C<T> a)
{
    T n = a.r * a.r + a.i * a.i;
    T s = rcp(n);
    return {a.r * s, -a.i * s};
}

__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tatan2(float y, float x) { return atan2f(y, x); }
__device__ __forceinline__ double tatan2(double y, double x) { return atan2(y, x); }
__device__ __forceinline__ float tlog(float x) { return logf(x); }
__device__ __forceinline__ double tlog(double x) { return log(x); }

// principal square root
template <typename T>
__device__ __forceinline__ C<T> csqrt_p(C<T> z)
{
    T m = tsqrt(z.r * z.r + z.i * z.i);
    if (m == T(0)) return {T(0), T(0)};
    if (z.r >= T(0)) {
        T u = tsqrt(T(0.5) * (m + z.r));
        return {u, z.i / (T(2) * u)};
    }
    T v = tsqrt(T(0.5) * (m - z.r));
    v = z.i < T(0) ? -v : v;
    return {z.i / (T(2) * v), v};
}

template <typename T>
__device__ __forceinline__ T cabs2(C<T> a) { return a.r * a.r + a.i * a.i; }
template <>
__device__ __forceinline__ df cabs2(C<df> a) { return fma(a.r, a.r, a.i * a.i); }
template <typename T>
__device__ __forceinline__ T cabs1(C<T> a) { return fabs(a.r) + fabs(a.i); }

// ----------------------------------------------------------------------------
// per-point contour plan (Step 3)
// ----------------------------------------------------------------------------
template <typename T>
struct Term {
    C<T> c;      // coefficient
    C<T> m2k;    // k-leg 1/(y + m2k) (ignored when full)
    C<T> m2q;    // (p-k)-leg mass: a = x + y + m2q
    int full;    // k-leg is the whole dressed propagator
};

template <typename T>
struct Plan {
    int npass;
    int kind[2];
    int nterm[2];
    Term<T> term[2][2];
    C<T> eth;    // e^{i arg(x)/2}: direction of the q-ray
    C<T> yp;     // pole passed by the detour
    int clus;    // clustered radial rule on the ray of pass 0
    double cl_c, cl_d, cl_eta;   // its centre c, width d and asinh(c/d)
};

template <typename T>
__device__ __forceinline__ C<T> cvt(double r, double i) { return {T(r), T(i)}; }

__device__ __forceinline__ double PI_D() { return 3.14159265358979323846; }

// distance from the y-ray along arg y = phi to the point y0
__device__ __forceinline__ double ray_distance(double y0r, double y0i, double phi)
{
    double d = fabs(atan2(y0i, y0r) - phi);
    if (d > PI_D()) d = 2.0 * PI_D() - d;
    return d < 0.5 * PI_D() ? sqrt(y0r * y0r + y0i * y0i) * sin(d) : sqrt(y0r * y0r + y0i * y0i);
}

// The plan is decided in binary64 (it selects among contours), then its
// numbers are rounded to T.
template <typename T, int CL = 0>
__device__ __forceinline__ Plan<T> make_plan(const KParams &kp, double xr, double xi)
{
    Plan<T> P;
    const PropConst &pc = kp.pc;
    // arg x decides the contour only for poles off the real axis
    const double phi = pc.kind == 0 ? 0.0 : atan2(xi, xr);
    double ax = sqrt(xr * xr + xi * xi);
    // e^{i phi/2} as the principal root of x/|x|: in binary64, or, for the
    // default binary32 kernels, x/|x| scaled in binary64 and its root (of
    // modulus 1) in binary32, whose pipes are 64 times faster; the sign of
    // Im x stays exact, so a point next to the cut keeps its side. (The
    // clustered radial rule of the variant kernels places its panels from
    // the binary64 direction.)
    C<double> eth = {1.0, 0.0};
    if constexpr (std::is_same<T, float>::value && !CL) {
        if (ax > 0.0) {
            const double ia = 1.0 / ax;
            const float ur = (float)(xr * ia), ui = (float)(xi * ia);
            C<float> e = csqrt_p(C<float>{ur, ui});
            if (ui == 0.0f && xi < 0.0) e.i = -e.i;
            P.eth = e;
        } else {
            P.eth = {1.0f, 0.0f};
        }
    } else {
        eth = csqrt_p(ax > 0.0 ? C<double>{xr / ax, xi / ax} : C<double>{1.0, 0.0});
        P.eth = cvt<T>(eth.r, eth.i);
    }
    P.clus = 0;
    P.cl_c = P.cl_d = P.cl_eta = 0.0;
    P.npass = 1;
    P.kind[0] = PASS_RAY;
    P.kind[1] = PASS_RAY;
    P.nterm[0] = 1;
    P.nterm[1] = 0;
    P.yp = {T(0), T(0)};
    if (pc.kind == 0) {                       // SCALAR
        Term<T> t;
        t.c = {T(1), T(0)};
        t.m2k = t.m2q = {T(pc.m2), T(0)};
        t.full = 0;
        P.term[0][0] = t;
    } else if (pc.kind == 1) {                // CPAIR
        // k-leg carries the pole in the half-plane of Im x; on the real axis
        // the legs stay as given (yu_* then holds the given k-leg pole)
        double ykr = pc.yu_re, yki = xi < 0.0 ? -pc.yu_im : pc.yu_im;
        if (xi == 0.0) { ykr = pc.yk0_re; yki = pc.yk0_im; }
        Term<T> t;
        t.c = {T(1), T(0)};
        t.m2k = cvt<T>(-ykr, -yki);
        t.m2q = cvt<T>(-ykr, yki);
        t.full = 0;
        P.term[0][0] = t;
        bool swept = xi != 0.0 && fabs(phi) > pc.arg_yu;
        bool graze = xi != 0.0 && ray_distance(ykr, yki, phi) < 2.0 * kp.r_detour;
        if (swept || graze) {
            P.kind[0] = PASS_DETOUR;
            P.yp = cvt<T>(ykr, yki);
        }
    } else {                                  // DRESSED
        C<double> yp = {pc.yp_re, pc.yp_im}, ym = {pc.yp_re, -pc.yp_im};
        C<double> Rp = {pc.Rp_re, pc.Rp_im}, Rm = {pc.Rp_re, -pc.Rp_im};
        if (fabs(phi) < pc.arg_yp) {
            // nothing swept: P(y) [P(s) - P(y)] on the ray, P(s) split in two
            P.nterm[0] = 2;
            P.term[0][0] = Term<T>{cvt<T>(Rp.r, Rp.i), {T(0), T(0)}, cvt<T>(-yp.r, -yp.i), 1};
            P.term[0][1] = Term<T>{cvt<T>(Rm.r, Rm.i), {T(0), T(0)}, cvt<T>(-ym.r, -ym.i), 1};
        } else {
            // partial fractions: the equal-pole terms on the ray (the one
            // whose pole lies in the half-plane of Im x on the opposite q-ray,
            // which flips the sign of the measure when D is odd), the mixed
            // term on the detour around the pole in the half-plane of Im x
            double sgn = (kp.dim & 1) ? -1.0 : 1.0;
            C<double> Rp2 = Rp * Rp, Rm2 = Rm * Rm;
            double sp = xi > 0.0 ? sgn : 1.0, sm = xi > 0.0 ? 1.0 : sgn;
            P.nterm[0] = 2;
            P.term[0][0] = Term<T>{cvt<T>(sp * Rp2.r, sp * Rp2.i), cvt<T>(-yp.r, -yp.i),
                                   cvt<T>(-yp.r, -yp.i), 0};
            P.term[0][1] = Term<T>{cvt<T>(sm * Rm2.r, sm * Rm2.i), cvt<T>(-ym.r, -ym.i),
                                   cvt<T>(-ym.r, -ym.i), 0};
            C<double> yk = xi > 0.0 ? yp : ym, yq = xi > 0.0 ? ym : yp;
            C<double> c2 = 2.0 * (Rp * Rm);
            P.npass = 2;
            P.kind[1] = PASS_DETOUR;
            P.nterm[1] = 1;
            P.term[1][0] = Term<T>{cvt<T>(c2.r, c2.i), cvt<T>(-yk.r, -yk.i),
                                   cvt<T>(-yq.r, -yq.i), 0};
            P.yp = cvt<T>(yk.r, yk.i);
        }
    }
    if (CL && kp.radial_rule == 1 && P.kind[0] == PASS_RAY) {
        // clustered radial rule: of the q-plane points +-sqrt(y_p) of the
        // propagator's poles, the one closest in angle to the ray, with
        // distance d < 0.75 of its projection c on the ray
        C<double> ys[2];
        int ny = 2;
        if (pc.kind == 0) { ys[0] = {-pc.m2, 0.0}; ny = 1; }
        else if (pc.kind == 1) { ys[0] = {pc.yu_re, pc.yu_im}; ys[1] = {pc.yu_re, -pc.yu_im}; }
        else { ys[0] = {pc.yp_re, pc.yp_im}; ys[1] = {pc.yp_re, -pc.yp_im}; }
        double best = 1.0;
        for (int i = 0; i < ny; ++i) {
            const C<double> z = csqrt_p(ys[i]) * conj(eth);
            for (int sg = -1; sg <= 1; sg += 2) {
                const double rs = sg * z.r, ds = fabs(z.i);
                if (rs > 0.0 && ds < 0.75 * rs && ds / rs < best) {
                    best = ds / rs;
                    P.clus = 1;
                    P.cl_c = rs;
                    P.cl_d = ds;
                }
            }
        }
        if (P.clus) {
            P.cl_d = fmax(P.cl_d, 1e-12 * P.cl_c);
            P.cl_eta = asinh(P.cl_c / P.cl_d);
        }
    }
    return P;
}

// Binary64 band of the mixed precision: points whose radial ray runs within
// pinch_angle of a direction where the angular integrand pinches, or that lie
// within cut_band of a branch-cut half-line on the real axis.
__device__ __forceinline__ bool in_band(const KParams &kp, double xr, double xi)
{
    const PropConst &pc = kp.pc;
    // squared distance to the half-line x <= thr against the squared band
    const double dr = xr <= pc.thr ? 0.0 : xr - pc.thr;
    if (dr * dr + xi * xi < kp.cut_band * kp.cut_band) return true;
    if (kp.pinch_angle > 0.0 && pc.pinch > 0.0 && fabs(fabs(atan2(xi, xr)) - pc.pinch) < kp.pinch_angle)
        return true;
    return false;
}

// ----------------------------------------------------------------------------
// nodes of the contour (Step 3) with the measure (1/2) y^((D-2)/2) dy
// ----------------------------------------------------------------------------
// Binary32 and double-float nodes carry their measure divided by (1 + |y|)^2
// and each of the two propagator fractions times (1 + |y|), so that neither
// overflows binary32's range far out on the contour; binary64 needs no such
// scaling and skips its reciprocal.
template <typename T>
__host__ __device__ constexpr bool node_scaled() { return !std::is_same<T, double>::value; }

template <typename T>
struct Node {
    C<T> y;
    C<T> Jt;    // measure, / (1 + |y|)^2 where node_scaled<T>()
    T sc;       // 1 + |y| where node_scaled<T>(), else 1
    C<T> ylo;   // binary32 ray nodes: y's rounding remainder (y = y + ylo exactly
                // for the node |q| = rho_hi + rho_lo on the ray e2); else 0
};

template <typename T>
__device__ __forceinline__ void load2(const KParams &kp, int which, int k, T &a, T &b);

template <>
__device__ __forceinline__ void load2<double>(const KParams &kp, int which, int k, double &a,
                                              double &b)
{
    const double2 *p = which == 0 ? kp.rad64 : (which == 1 ? kp.seg64 : (which == 2 ? kp.arc64 : kp.tail64));
    double2 v = __ldg(p + k);
    a = v.x;
    b = v.y;
}

template <>
__device__ __forceinline__ void load2<df>(const KParams &kp, int which, int k, df &a, df &b)
{
    const float4 *p = which == 0 ? kp.rad_df : (which == 1 ? kp.seg_df : (which == 2 ? kp.arc_df : kp.tail_df));
    float4 v = __ldg(p + k);
    a = df(v.x, v.y);
    b = df(v.z, v.w);
}

template <>
__device__ __forceinline__ void load2<float>(const KParams &kp, int which, int k, float &a,
                                             float &b)
{
    const float2 *p = which == 0 ? kp.rad32 : (which == 1 ? kp.seg32 : (which == 2 ? kp.arc32 : kp.tail32));
    float2 v = __ldg(p + k);
    a = v.x;
    b = v.y;
}

// q-ray node at |q| = rho with weight W: q = rho e^{i theta}, y = rho^2
// e^{2 i theta} (e2), measure q^(D-1) dq
template <typename T>
__device__ __forceinline__ Node<T> ray_node_at(const KParams &kp, T rho, T W, C<T> e2, C<T> eD)
{
    Node<T> n;
    const T r2 = rho * rho;
    n.y = r2 * e2;
    // q^(D-1) e^{i theta} = rho^(D-1) e^{i D theta}
    T mag;
    if constexpr (node_scaled<T>()) {
        // rho^(D-1) W / (1 + rho^2)^2, scaled first so binary32 cannot overflow
        n.sc = T(1) + r2;
        T s = rcp(n.sc);
        s = s * s;
        const T rs = r2 * s;
        mag = (kp.dim == 4 ? rs * rho : rs) * W;
    } else {
        n.sc = T(1);
        mag = (kp.dim == 4 ? r2 * rho : r2) * W;
    }
    n.Jt = mag * eD;
    return n;
}

// node k of the mapped ray from q = 0 (binary64: rho^2 and the measure
// rho^(D-1) W from the table, rounded there as ray_node_at rounds them)
template <typename T>
__device__ __forceinline__ Node<T> ray_node(const KParams &kp, int k, C<T> e2, C<T> eD)
{
    if constexpr (std::is_same<T, double>::value) {
        const double2 v = __ldg(kp.rayp64 + k);
        Node<T> n;
        n.y = v.x * e2;
        n.sc = 1.0;
        n.Jt = v.y * eD;
        n.ylo = {0.0, 0.0};
        return n;
    } else {
        T rho, W;
        load2<T>(kp, 0, k, rho, W);
        Node<T> n = ray_node_at<T>(kp, rho, W, e2, eD);
        n.ylo = {T(0), T(0)};
        return n;
    }
}

// node k of the mapped ray from |q| = rho0 > 0 (the tail of a detour)
template <typename T>
__device__ __forceinline__ Node<T> ray_node_from(const KParams &kp, int k, C<T> e2, C<T> eD,
                                                 T rho0)
{
    T rho, W;
    load2<T>(kp, 0, k, rho, W);
    Node<T> n = ray_node_at<T>(kp, rho + rho0, W, e2, eD);
    n.ylo = {T(0), T(0)};
    return n;
}

// binary32 node k of the ray from q = 0, with y exact: |q| = rho_hi + rho_lo
// from the double-float table, rho^2 = p + pe by an FMA TwoProduct, and
// y = p e2 + pe e2 split into its rounded value and remainder (TwoProduct
// again), so that y + M2 and a = x + y + M2 can be formed with one rounding
// each (the contour passes close to y = -M2 next to the negative real axis,
// where y + M2 cancels).
__device__ __forceinline__ Node<float> ray_node_exact_y(const KParams &kp, int k, C<float> e2,
                                                        C<float> eD, C<float> e2lo = {0.0f, 0.0f})
{
    const float4 v = __ldg(kp.rad_df + k);
    const float rh = v.x, rl = v.y, W = v.z;
    const float p = rh * rh;
    const float pe = fmaf(rh, rh, -p) + 2.0f * rh * rl;
    Node<float> n;
    n.y.r = p * e2.r;
    n.y.i = p * e2.i;
    // (with e2lo, the ray direction's own remainder: the ray of the exact
    // direction x/|x|, not of its binary32 rounding)
    n.ylo.r = fmaf(p, e2lo.r, fmaf(p, e2.r, -n.y.r) + pe * e2.r);
    n.ylo.i = fmaf(p, e2lo.i, fmaf(p, e2.i, -n.y.i) + pe * e2.i);
    n.sc = 1.0f + p;
    float s = rcp(n.sc);
    s = s * s;
    const float rs = p * s;
    n.Jt = ((kp.dim == 4 ? rs * rh : rs) * W) * eD;
    return n;
}

// node k of the clustered ray: n_s nodes on [0, c] and on [c, 2c] with
// |q| = c + d sinh(s), s = eta (t - 1) or eta t, dq = d cosh(s) eta dt, then
// the n_r/2 tail nodes from 2c
__device__ __forceinline__ void cl_rho_w(const KParams &kp, int k, double c, double d,
                                         double eta, double &rho, double &W)
{
    const int ns = kp.n_s;
    if (k < 2 * ns) {
        double t, w;
        load2<double>(kp, 1, k < ns ? k : k - ns, t, w);
        const double sv = k < ns ? eta * (t - 1.0) : eta * t;
        const double e = exp(sv), ie = rcp(e);
        rho = c + d * (0.5 * (e - ie));
        W = d * (0.5 * (e + ie)) * eta * w;
    } else {
        double rt, wt;
        load2<double>(kp, 3, k - 2 * ns, rt, wt);
        rho = 2.0 * c + rt;
        W = wt;
    }
}
__device__ __forceinline__ void cl_rho_w(const KParams &kp, int k, double c, double d,
                                         double eta, float &rho, float &W)
{
    const int ns = kp.n_s;
    if (k < 2 * ns) {
        float t, w;
        load2<float>(kp, 1, k < ns ? k : k - ns, t, w);
        const float sv = k < ns ? (float)eta * (t - 1.0f) : (float)eta * t;
        const float e = expf(sv), ie = rcp(e);
        rho = (float)c + (float)d * (0.5f * (e - ie));
        W = (float)d * (0.5f * (e + ie)) * (float)eta * w;
    } else {
        float rt, wt;
        load2<float>(kp, 3, k - 2 * ns, rt, wt);
        rho = 2.0f * (float)c + rt;
        W = wt;
    }
}
__device__ __forceinline__ void cl_rho_w(const KParams &kp, int k, double c, double d,
                                         double eta, df &rho, df &W)
{
    double r, w;
    cl_rho_w(kp, k, c, d, eta, r, w);
    rho = df(r);
    W = df(w);
}

template <typename T>
__device__ __forceinline__ Node<T> ray_node_cl(const KParams &kp, int k, C<T> e2, C<T> eD,
                                               double c, double d, double eta)
{
    T rho, W;
    cl_rho_w(kp, k, c, d, eta, rho, W);
    Node<T> n = ray_node_at<T>(kp, rho, W, e2, eD);
    n.ylo = {T(0), T(0)};
    return n;
}

template <typename T>
__device__ __forceinline__ C<T> half_pow(const KParams &kp, C<T> y)
{
    // (1/2) y^((D-2)/2): D = 4 -> y/2, D = 3 -> sqrt(y)/2 (principal)
    if (kp.dim == 4) return T(0.5) * y;
    return T(0.5) * csqrt_p(y);
}

template <typename T>
__device__ __forceinline__ Node<T> finish_y_node(const KParams &kp, C<T> y, C<T> dy)
{
    Node<T> n;
    n.y = y;
    n.ylo = {T(0), T(0)};
    n.Jt = half_pow(kp, y) * dy;
    if constexpr (node_scaled<T>()) {
        n.sc = T(1) + tsqrt(cabs2(y));
        T s = rcp(n.sc);
        n.Jt = (s * s) * n.Jt;
    } else {
        n.sc = T(1);
    }
    return n;
}

// Per-pass constants of a detour around the pole yp (computed once per point)
template <typename T>
struct DetourPre {
    C<T> yp, u, q1, y0, d;   // pole, yp/|yp|, end of the q-segment, outer segment y0 -> y0 + d
    T r, sqRd, sgpr, sg;     // radius, sqrt(R_d), sign(Im yp) pi r, sign(Im yp)
};

template <typename T>
__device__ __forceinline__ DetourPre<T> detour_pre(const KParams &kp, C<T> eth, C<T> yp, C<T> x)
{
    DetourPre<T> dp;
    const T ap = tsqrt(cabs2(yp));
    dp.yp = yp;
    dp.u = rcp(ap) * yp;
    dp.r = T(kp.r_detour);
    const T Rd = tsqrt(cabs2(x)) + T(20);
    dp.sqRd = tsqrt(Rd);
    dp.q1 = csqrt_p((ap - dp.r) * dp.u);
    dp.y0 = (ap + dp.r) * dp.u;
    dp.d = Rd * (eth * eth) - dp.y0;
    dp.sg = yp.i > T(0) ? T(1) : T(-1);
    dp.sgpr = dp.sg * T(PI_D()) * dp.r;
    return dp;
}

// A warp's DetourPre lives in shared memory (one slot per warp of a block of
// 256): held in registers across the node loop it raised the register count
// of every kernel, ray-only ones included.
template <typename T>
__device__ __forceinline__ DetourPre<T> *detour_slot()
{
    __shared__ DetourPre<T> slots[8];
    return &slots[threadIdx.x >> 5];
}

// detour node k of 3 n_s + n_r: q-segment 0 -> q1, half circle around yp,
// straight segment out to R_d e^{i phi}, ray to infinity from |q| = sqrt(R_d)
template <typename T>
__device__ __forceinline__ Node<T> detour_node(const KParams &kp, int k, C<T> e2, C<T> eD,
                                               const DetourPre<T> &dp)
{
    const int ns = kp.n_s;
    if (k >= 3 * ns) return ray_node_from<T>(kp, k - 3 * ns, e2, eD, dp.sqRd);
    T t, w;
    if (k < ns) {
        load2<T>(kp, 1, k, t, w);
        const C<T> q1 = dp.q1;
        C<T> q = t * q1;
        Node<T> n;
        n.y = q * q;
        n.ylo = {T(0), T(0)};
        // measure q^(D-1) dq, dq = q1 w
        C<T> qd = kp.dim == 4 ? q * q * q : q * q;
        n.Jt = w * (qd * q1);
        if constexpr (node_scaled<T>()) {
            n.sc = T(1) + cabs2(q);
            T s = rcp(n.sc);
            n.Jt = (s * s) * n.Jt;
        } else {
            n.sc = T(1);
        }
        return n;
    }
    if (k < 2 * ns) {
        load2<T>(kp, 1, k - ns, t, w);
        T cs, sn;
        load2<T>(kp, 2, k - ns, cs, sn);
        // theta = th0 + sg pi t with e^{i th0} = -u, sg = sign(Im yp)
        C<T> e = cx<T>(-dp.u.r, -dp.u.i) * cx<T>(cs, dp.sg * sn);
        C<T> y = dp.yp + dp.r * e;
        C<T> dy = (dp.sgpr * w) * cx<T>(-e.i, e.r);   // i r e dtheta
        return finish_y_node<T>(kp, y, dy);
    }
    load2<T>(kp, 1, k - 2 * ns, t, w);
    return finish_y_node<T>(kp, dp.y0 + t * dp.d, w * dp.d);
}

// ----------------------------------------------------------------------------
// angular pair sum
// ----------------------------------------------------------------------------
// |1 - w t|^2 for one angular node. Direct form (1 - wr t)^2 + (wi t)^2: its
// rounding error relative to the result is ~ eps/|1 - w t| next to a pinch.
// Horner form 1 + t (|w|^2 t - 2 wr): two FMAs, error ~ eps/|1 - w t|^2, used
// only for compressed rules, whose selection keeps |1 - w t| away from zero.
__device__ __forceinline__ double q_direct(double t, double wr, double wi)
{
    double dr = fma(-wr, t, 1.0);
    double di = wi * t;
    return fma(dr, dr, di * di);
}
__device__ __forceinline__ float q_direct(float t, float wr, float wi)
{
    float dr = fmaf(-wr, t, 1.0f);
    float di = wi * t;
    // keep the reciprocal finite if rounding lands on zero at a pinch
    return fmaxf(fmaf(dr, dr, di * di), 1e-30f);
}
__device__ __forceinline__ df q_direct(df t, df wr, df wi)
{
    df dr = fma(-wr, t, df(1));
    df di = wi * t;
    return fma(dr, dr, di * di);
}
// s += e r for the positive angular sums A and B; double-float accumulates
// unnormalised (cascaded summation) and pos_finish renormalises once
__device__ __forceinline__ void pos_acc(float &s, float e, float r) { s = fmaf(e, r, s); }
__device__ __forceinline__ void pos_acc(double &s, double e, double r) { s = fma(e, r, s); }
__device__ __forceinline__ float pos_finish(float s) { return s; }
__device__ __forceinline__ double pos_finish(double s) { return s; }

template <typename T>
__device__ __forceinline__ T q_horner(T t, T w2, T m2wr)
{
    return fma(fma(w2, t, m2wr), t, T(1));
}

// Where the pole t = 1/w of 1/(1 - w t) lies relative to the interval [0, 1]:
// on the Bernstein ellipse of parameter rho >= 1, i.e. the ellipse with foci
// t = 0 and t = 1 through 1/w, whose distances to the foci sum to
// (rho + 1/rho)/2 in units of the interval. That sum is
//   sigma = (|1/w| + |1/w - 1|) = (1 + |1 - w|) / |w|,
// monotone in rho, so the rule thresholds are compared in sigma. Two
// reciprocal square roots (the hardware approximations: the thresholds carry
// a factor 10 of margin in the error they bound); w = 0 gives infinity (the
// smallest rule), a pole on the interval (w = 1/t) 1/|w| <= 1 (the full table).
__device__ __forceinline__ float sigma_of(float wr, float wi)
{
    const float n2 = wr * wr + wi * wi;
    if (!(n2 > 0.0f)) return __int_as_float(0x7f800000);
    const float dr = 1.0f - wr;
    const float q = fmaxf(fmaf(dr, dr, wi * wi), 1e-30f);
    return fmaf(q, rsqrtf(q), 1.0f) * rsqrtf(n2);
}

// An approximate binary32 value for the rule selection: binary32 as is, the
// high part of a double-float, and binary64 truncated by integer operations
// on its bits (relative error below 2^-23; a conversion instruction would
// occupy the FP64 pipe, which bounds the binary64 kernel). Magnitudes below
// binary32's normal range give 0, above it infinity.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(df v) { return v.hi; }
__device__ __forceinline__ float to_f32(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
    const unsigned sign = hi & 0x80000000u;
    if (e <= 0) return __int_as_float((int)sign);
    if (e >= 255) return __int_as_float((int)(sign | 0x7f800000u));
    return __int_as_float((int)(sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29)));
}

template <typename T>
__device__ __forceinline__ float sig_min(const KParams &kp, int r);
template <>
__device__ __forceinline__ float sig_min<float>(const KParams &kp, int r) { return kp.sig_min32[r]; }
template <>
__device__ __forceinline__ float sig_min<double>(const KParams &kp, int r) { return kp.sig_min64[r]; }
template <>
__device__ __forceinline__ float sig_min<df>(const KParams &kp, int r) { return kp.sig_min64[r]; }

// one node (tau, gamma, gamma tau) of a compressed rule in shared memory
__device__ __forceinline__ void rule_node(const void *srules, int k, double &t, double &e,
                                          double &g)
{
    const double *p = reinterpret_cast<const double *>(srules) + 3 * k;
    t = p[0];
    e = p[1];
    g = p[2];
}
__device__ __forceinline__ void rule_node(const void *srules, int k, df &t, df &e, df &g)
{
    const float2 *p = reinterpret_cast<const float2 *>(srules) + 3 * k;
    t = df(p[0].x, p[0].y);
    e = df(p[1].x, p[1].y);
    g = df(p[2].x, p[2].y);
}
__device__ __forceinline__ void rule_node(const void *srules, int k, float &t, float &e, float &g)
{
    float4 v = reinterpret_cast<const float4 *>(srules)[k];
    t = v.x;
    e = v.y;
    g = v.z;
}

// Unroll factors of the runtime-length angular pair loops. Double-float
// bodies are several times larger than binary64 ones; unrolled they no longer
// fit the instruction cache (measured on GB300, production bubble grid:
// unroll 4 / 2 / 1 gives 2.95 / 3.74 / 4.06 Mpoints/s in double-float).
#ifndef GFC_DF_UNROLL
#define GFC_DF_UNROLL 1
#endif
#ifndef GFC_F32_UNROLL
#define GFC_F32_UNROLL 4
#endif
template <typename T>
__host__ __device__ constexpr int pair_unroll()
{
    return std::is_same<T, df>::value ? GFC_DF_UNROLL
                                      : (std::is_same<T, float>::value ? GFC_F32_UNROLL : 4);
}

// Angular sums A = sum e_j/q_j, B = sum g_j/q_j for NT terms; qmin (binary32
// only) is the smallest q met, a measure of how close the node is to a pinch.
template <typename T, int NP, int NT>
__device__ __forceinline__ int pair_sums(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                         int npair, const T *stab, const void *srules,
                                         const C<T> (&w)[NT], T (&A)[NT], T (&B)[NT], T &qmin)
{
    constexpr bool f32 = sizeof(T) == 4;
    T w2[NT], m2wr[NT], A1[NT], B1[NT];
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        w2[s] = cabs2(w[s]);
        m2wr[s] = T(-2) * w[s].r;
        A[s] = B[s] = A1[s] = B1[s] = T(0);
    }
    T qm = T(1e30);
    // the smallest compressed rule that is exact to rounding level for every
    // term, made uniform over the lanes that run together
    int rule = kp.nrule;
    {
        float sig = __int_as_float(0x7f800000);
#pragma unroll
        for (int s = 0; s < NT; ++s) sig = fminf(sig, sigma_of(to_f32(w[s].r), to_f32(w[s].i)));
        // rho from sigma = (rho + 1/rho)/2 (2 sigma beyond 1e4, and for an
        // infinite sigma); the rule needs rule_n >= K/ln(rho), taken 1e-4
        // larger: the approximate square root, logarithm and reciprocal
        // carry relative errors of a few 1e-7 in K/ln(rho) wherever it is
        // below 127 (ln(rho) >= 0.08); a NaN selects the full table
        const float s2m1 = fmaxf(fmaf(sig, sig, -1.0f), 0.0f);
        const float rho = sig > 1e4f ? 2.0f * sig : sig + s2m1 * rsqrtf(fmaxf(s2m1, 1e-30f));
        const float nstar = (std::is_same<T, float>::value ? kp.rule_k32 : kp.rule_k64) * 1.0001f *
                            rcp(__logf(rho));
        rule = nstar < 127.0f ? (int)kp.rule_idx[(int)ceilf(fmaxf(nstar, 0.0f))] : kp.nrule;
        rule = __reduce_max_sync(__activemask(), rule);
    }
    if (rule < kp.nrule) {
        const int off = kp.rule_off[rule], n = kp.rule_n[rule];
#pragma unroll (pair_unroll<T>())
        for (int k = 0; k < n; ++k) {
            T t, e, g;
            rule_node(srules, off + k, t, e, g);
#pragma unroll
            for (int s = 0; s < NT; ++s) {
                T q = f32 ? q_direct(t, w[s].r, w[s].i) : q_horner(t, w2[s], m2wr[s]);
                if (f32) qm = fmin(qm, q);
                T r = rcp(q);
                pos_acc(A[s], e, r);
                pos_acc(B[s], g, r);
            }
        }
    } else if (NP > 0) {
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            const T t = tab.t[j], e = tab.e[j], g = tab.g[j];
#pragma unroll
            for (int s = 0; s < NT; ++s) {
                T q = q_direct(t, w[s].r, w[s].i);
                if (f32) qm = fmin(qm, q);
                T r = rcp(q);
                if (j & 1) {
                    pos_acc(A1[s], e, r);
                    pos_acc(B1[s], g, r);
                } else {
                    pos_acc(A[s], e, r);
                    pos_acc(B[s], g, r);
                }
            }
        }
#pragma unroll
        for (int s = 0; s < NT; ++s) {
            A[s] = pos_finish(A[s]) + pos_finish(A1[s]);
            B[s] = pos_finish(B[s]) + pos_finish(B1[s]);
        }
    } else {
#pragma unroll (pair_unroll<T>())
        for (int j = 0; j < npair; ++j) {
            const T t = stab[3 * j], e = stab[3 * j + 1], g = stab[3 * j + 2];
#pragma unroll
            for (int s = 0; s < NT; ++s) {
                T q = q_direct(t, w[s].r, w[s].i);
                if (f32) qm = fmin(qm, q);
                T r = rcp(q);
                pos_acc(A[s], e, r);
                pos_acc(B[s], g, r);
            }
        }
    }
    if (rule < kp.nrule || NP == 0) {
#pragma unroll
        for (int s = 0; s < NT; ++s) {
            A[s] = pos_finish(A[s]);
            B[s] = pos_finish(B[s]);
        }
    }
    qmin = qm;
    // pairs evaluated; negative when they were the full table's
    return rule < kp.nrule ? kp.rule_n[rule] : -npair;
}

// The angular integral in closed form, the limit of every angular rule: half
// of int_0^pi sin^(D-2) psi (v c - 1)/(1 - w c) dpsi, c = cos^2 psi (the half
// matches the pair sums, which weight each +-psi pair once). With
// (v c - 1)/(1 - w c) = -v/w + (v/w - 1)/(1 - w c):
//   D = 4: int sin^2/(1 - w c) = pi/(1 + s), s = sqrt(1 - w), and the whole
//          reduces to (pi/2)(v/(2(1 + s)) - 1)/(1 + s), free of cancellation;
//   D = 3: int sin/(1 - w c) = 2 A, A = artanh(sqrt w)/sqrt w, giving
//          (v - w) B1 - 1 with B1 = (A - 1)/w = sum_k>=1 w^(k-1)/(2k + 1)
//          (the series for |w| < 0.1, the logarithms otherwise).
// Principal branches: analytic off w in [1, inf), where the angular
// integrand has its poles; the contours keep w off that half-line.
template <typename T>
__device__ __forceinline__ C<T> exact_S4(C<T> v, C<T> w)
{
    const T one = T(1);
    C<T> s = csqrt_p(C<T>{one - w.r, -w.i});
    C<T> r = cinv(C<T>{one + s.r, s.i});
    C<T> u = T(0.5) * (v * r);
    return T(0.5 * PI_D()) * (C<T>{u.r - one, u.i} * r);
}
template <typename T>
__device__ __forceinline__ C<T> exact_S_impl(int dim, C<T> v, C<T> w)
{
    const T one = T(1);
    if (dim == 4) return exact_S4<T>(v, w);
    C<T> B1;
    if (cabs2(w) < T(0.01)) {
        // sum_k>=1 w^(k-1)/(2k + 1) to rounding level for |w| < 0.1
        B1 = C<T>{T(1.0 / 37.0), T(0)};
        for (int k = 17; k >= 1; --k) B1 = C<T>{T(1) / T(2 * k + 1), T(0)} + w * B1;
    } else {
        C<T> z = csqrt_p(w);
        // artanh z = (log(1 + z) - log(1 - z))/2, principal logarithms
        C<T> p = {one + z.r, z.i}, m = {one - z.r, -z.i};
        T lr = T(0.5) * (tlog(cabs2(p)) - tlog(cabs2(m)));
        T li = tatan2(p.i, p.r) - tatan2(m.i, m.r);
        C<T> at = T(0.5) * C<T>{lr, li};
        C<T> A = at * cinv(z);
        B1 = C<T>{A.r - one, A.i} * cinv(w);
    }
    C<T> vw = v - w;
    C<T> r = vw * B1;
    return C<T>{r.r - one, r.i};
}
template <typename T>
__device__ __forceinline__ C<T> exact_S(int dim, C<T> v, C<T> w) { return exact_S_impl<T>(dim, v, w); }
// double-float: D = 4 natively; D = 3 (logarithms) evaluated in binary64
template <>
__device__ __forceinline__ C<df> exact_S<df>(int dim, C<df> v, C<df> w)
{
    if (dim == 4) return exact_S4<df>(v, w);
    C<double> r = exact_S_impl<double>(dim, C<double>{(double)v.r, (double)v.i},
                                       C<double>{(double)w.r, (double)w.i});
    return C<df>{df(r.r), df(r.i)};
}

// Omega1, delta and the dressed pole and residue as T, read from the kernel
// parameters (constant-bank operands): binary64 from the binary64 fields,
// the other arithmetics from copies the host stores in their own type, so
// that no node converts binary64 on the FP64 pipe.
template <typename T>
struct KConst;
template <>
struct KConst<double> {
    static __device__ __forceinline__ double om1(const KParams &kp) { return kp.Omega1; }
    static __device__ __forceinline__ double del(const KParams &kp) { return kp.delta; }
    static __device__ __forceinline__ C<double> yp(const KParams &kp) { return {kp.pc.yp_re, kp.pc.yp_im}; }
    static __device__ __forceinline__ C<double> Rp(const KParams &kp) { return {kp.pc.Rp_re, kp.pc.Rp_im}; }
};
template <>
struct KConst<float> {
    static __device__ __forceinline__ float om1(const KParams &kp) { return kp.f32c[0]; }
    static __device__ __forceinline__ float del(const KParams &kp) { return kp.f32c[1]; }
    static __device__ __forceinline__ C<float> yp(const KParams &kp) { return {kp.f32c[2], kp.f32c[3]}; }
    static __device__ __forceinline__ C<float> Rp(const KParams &kp) { return {kp.f32c[4], kp.f32c[5]}; }
};
template <>
struct KConst<df> {
    static __device__ __forceinline__ df g(const KParams &kp, int i) { return df(kp.dfc[2 * i], kp.dfc[2 * i + 1]); }
    static __device__ __forceinline__ df om1(const KParams &kp) { return g(kp, 0); }
    static __device__ __forceinline__ df del(const KParams &kp) { return g(kp, 1); }
    static __device__ __forceinline__ C<df> yp(const KParams &kp) { return {g(kp, 2), g(kp, 3)}; }
    static __device__ __forceinline__ C<df> Rp(const KParams &kp) { return {g(kp, 4), g(kp, 5)}; }
};

// Per-pass constants of one point, computed once and reused for every node.
template <typename T, int NT>
struct PassPre {
    int nt;
    C<T> m2q[NT], m2k[NT];
    C<T> cx2[NT];     // c_t 2x
    C<T> omx[NT];     // Omega (x + M2_t)
    int full[NT];     // k-leg is the whole dressed propagator
    int same[NT];     // k-leg and (p-k)-leg share the pole: one reciprocal
    C<T> xm[NT], xml[NT];   // x + M2_t rounded (binary32: and its remainder, TwoSum)
    C<T> x4;                // 4 x
    C<T> omxl[NT];          // binary32: Omega (x + M2_t) - omx (the product in binary64)
    C<T> xlo;               // binary32 with partial routing: x less its binary32 value
};



template <typename T, int NT, int ACC = 0>
__device__ __forceinline__ PassPre<T, NT> pass_pre(const KParams &kp, const Plan<T> &P, int pass,
                                                   C<T> x, C<T> xlo = {T(0), T(0)})
{
    PassPre<T, NT> pp;
    pp.xlo = xlo;
    pp.nt = P.nterm[pass];
    pp.x4 = T(4) * x;
    const T Om = T(kp.Omega);
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        const Term<T> &tm = P.term[pass][s < pp.nt ? s : 0];
        pp.m2q[s] = tm.m2q;
        pp.m2k[s] = tm.m2k;
        pp.cx2[s] = tm.c * (T(2) * x);
        if constexpr (!(std::is_same<T, float>::value && ACC)) pp.omx[s] = Om * (x + tm.m2q);
        pp.full[s] = tm.full;
        pp.same[s] = !tm.full && tm.m2k.r == tm.m2q.r && tm.m2k.i == tm.m2q.i;
        if constexpr (std::is_same<T, float>::value) {
            // TwoSum (Knuth): x + M2 = xm + xml exactly
            const C<T> m = tm.m2q;
            const T sr = x.r + m.r, si = x.i + m.i;
            const T br = sr - x.r, bi = si - x.i;
            pp.xm[s] = {sr, si};
            pp.xml[s] = {(x.r - (sr - br)) + (m.r - br), (x.i - (si - bi)) + (m.i - bi)};
        }
        if constexpr (std::is_same<T, float>::value && ACC) {
            // Omega (x + M2) to double-float accuracy, in binary32 operations
            // (TwoProduct of the high parts, the low terms gathered): rounded
            // once per pass it would shift every node's leading term alike
            // (see node_value). The asm keeps the four values in registers:
            // the compiler would otherwise recompute them per node.
            // x + M2 = xm + xml with x's own remainder (x less its binary32
            // value) in xml: every node's a = x + y + M2 then holds x to
            // double-float accuracy
            pp.xml[s] = pp.xml[s] + xlo;
            const float oh = kp.om_df[0], ol = kp.om_df[1];
            float pr = oh * pp.xm[s].r, pi = oh * pp.xm[s].i;
            float er = fmaf(oh, pp.xm[s].r, -pr) + (oh * pp.xml[s].r + ol * pp.xm[s].r);
            float ei = fmaf(oh, pp.xm[s].i, -pi) + (oh * pp.xml[s].i + ol * pp.xm[s].i);
            asm volatile("" : "+f"(pr), "+f"(pi), "+f"(er), "+f"(ei));
            pp.omx[s] = {pr, pi};
            pp.omxl[s] = {er, ei};
        }
    }
    return pp;
}

// Rounding-error scale of a point's binary32 sum, accumulated per lane: s1 =
// sum_k M_k, s2 = sum_k (M_k kappa_k)^2, with M_k = |v_k|_1 the magnitude of
// node k's contribution and kappa_k its relative condition number (below).
// Rounding errors of different nodes are independent, so they add like a
// root-sum-square (s2); s1 covers what all nodes share (the rounded per-point
// and rule constants).
template <typename T>
struct ErrAcc {
    T s1, s2;
};

__device__ __forceinline__ float trsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double trsqrt(double x) { return rsqrt(x); }
__device__ __forceinline__ df trsqrt(df x) { return df(rsqrtf(x.hi), 0.0f); }

// Contribution of one node of one pass: Jt * sum_t c_t P1_t(y)/(y + M2_t) *
// 2x/a_t * S_t, with the (1 + |y|)^2 scale (node_scaled) moved from Jt onto
// the fractions. With FC (one term) the pass's common factor c 2x is left out,
// for the caller to apply once to the pass's sum.
// The node's error scale is added to `ea` (binary32, and binary64 with cond
// output); `qmin` receives the smallest |1 - w t|^2 of its angular sums
// (binary32); `npairs` the angular pairs evaluated, negated when they were
// the full table's.
//
// kappa_k, the relative sensitivity of the node's value to rounding of its
// inputs: |y|/|y + M2| per propagator factor (the contour passes near a pole
// when arg x is near pi), (|x| + |y|)/|a| for the denominator a, and
// |w|/|1 - w t|_min for the angular sum next to a pinch (binary32 only).
template <typename T, int NP, int NT, int V, int FC = 0, int ACC = 0>
__device__ __forceinline__ C<T> node_value(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                           const T *stab, const void *srules,
                                           const PassPre<T, NT> &pp, C<T> x, const Node<T> &nd,
                                           ErrAcc<T> &ea, T &qmin, int &npairs, bool exact_y)
{
    constexpr bool f32 = std::is_same<T, float>::value;
    // y + c formed with one rounding from y's remainder (binary32), else plain
    auto ypc = [&](C<T> c) -> C<T> {
        if constexpr (f32) return C<T>{(nd.y.r + c.r) + nd.ylo.r, (nd.y.i + c.i) + nd.ylo.i};
        else return nd.y + c;
    };
    // (1 + |y|)/c where the node is scaled, else 1/c
    auto sinv = [&](C<T> c) -> C<T> {
        if constexpr (node_scaled<T>()) return nd.sc * cinv(c);
        else return cinv(c);
    };
    static_assert(!FC || NT == 1, "c 2x is common to the pass only for one term");
    // double-float has no error-scale output (it would cost registers)
    const bool want_mag = std::is_same<T, float>::value ||
                          (std::is_same<T, double>::value && kp.cond_out != nullptr);
    // u = y/a (v = 4u), w = 4xy/a^2
    C<T> ia[NT], u[NT], w[NT];
    T kap[NT];
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        C<T> a;
        if constexpr (f32)
            a = {(pp.xm[s].r + nd.y.r) + (pp.xml[s].r + nd.ylo.r),
                 (pp.xm[s].i + nd.y.i) + (pp.xml[s].i + nd.ylo.i)};
        else
            a = x + nd.y + pp.m2q[s];
        ia[s] = cinv(a);
        if constexpr (f32) {
            // binary32 keeps v = 4u itself (its registers are the scarcer)
            u[s] = T(4) * (nd.y * ia[s]);
            if constexpr (ACC) {
                // w = x v / a with x to double-float accuracy (x + its remainder)
                const C<T> xv = x * u[s], lv = pp.xlo * u[s];
                w[s] = C<T>{xv.r + lv.r, xv.i + lv.i} * ia[s];
            } else {
                w[s] = (x * u[s]) * ia[s];
            }
        } else {
            u[s] = nd.y * ia[s];
            w[s] = (pp.x4 * u[s]) * ia[s];
        }
        if (want_mag) kap[s] = (cabs1(x) + cabs1(nd.y)) * rcp(cabs1(a));
    }
    T A[NT], B[NT];
    C<T> Sx[NT];
    if (V && kp.ang_exact) {
        qmin = T(1e30);
#pragma unroll
        for (int s = 0; s < NT; ++s) {
            Sx[s] = exact_S<T>(kp.dim, f32 ? u[s] : T(4) * u[s], w[s]);
            if (sizeof(T) == 4) qmin = fmin(qmin, cabs2(C<T>{T(1) - w[s].r, -w[s].i}));
            A[s] = B[s] = T(0);
        }
        npairs = 0;
    } else {
        npairs = pair_sums<T, NP, NT>(kp, tab, kp.npair, stab, srules, w, A, B, qmin) * pp.nt;
    }
    const T Om1 = KConst<T>::om1(kp), del = KConst<T>::del(kp);
    C<T> sum = {T(0), T(0)};
    T mag = T(0), magk = T(0);
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        if (s >= pp.nt) break;
        C<T> S;
        if (V && kp.ang_exact) {
            S = Sx[s];
        } else {
            C<T> T2 = {A[s] - w[s].r * B[s], w[s].i * B[s]};
            C<T> lead;
            if constexpr (f32 && ACC) {
                // the leading term with its constants delta, Omega1 and
                // Omega (x + M2) to double-float accuracy (low parts from the
                // double-float copies): rounded to binary32 they would shift
                // every node's leading term alike, an error that cancels in a
                // sum over all nodes but not when some of them are evaluated
                // again in another arithmetic (partial routing)
                const float dl = kp.dfc[3], o1l = kp.dfc[1];
                const C<T> dy = {fmaf(del, nd.y.r, dl * nd.y.r), fmaf(del, nd.y.i, dl * nd.y.i)};
                const C<T> tt = {(dy.r - pp.omx[s].r) - pp.omxl[s].r, (dy.i - pp.omx[s].i) - pp.omxl[s].i};
                const C<T> ow = {fmaf(Om1, w[s].r, o1l * w[s].r), fmaf(Om1, w[s].i, o1l * w[s].i)};
                lead = tt * ia[s] - ow;
            } else {
                lead = (del * nd.y - pp.omx[s]) * ia[s] - Om1 * w[s];
            }
            // (v - w) w, v - w = 4u - w with one rounding
            const C<T> vmw = f32 ? u[s] - w[s]
                                 : C<T>{fma(T(4), u[s].r, -w[s].r), fma(T(4), u[s].i, -w[s].i)};
            const C<T> vw = vmw * w[s];
            S = lead + vw * T2;
        }
        // P1(y) / (y + M2), times (1 + |y|)^2 where the node is scaled
        const C<T> ypq = ypc(pp.m2q[s]);
        C<T> pq = sinv(ypq);
        C<T> p1;
        if (pp.same[s]) {
            p1 = pq;
        } else if (pp.full[s]) {
            const C<T> yp = KConst<T>::yp(kp), Rp = KConst<T>::Rp(kp);
            const C<T> pf = Rp * cinv(ypc(C<T>{-yp.r, -yp.i})) + conj(Rp) * cinv(ypc(C<T>{-yp.r, yp.i}));
            if constexpr (node_scaled<T>()) p1 = nd.sc * pf;
            else p1 = pf;
        } else {
            p1 = sinv(ypc(pp.m2k[s]));
        }
        C<T> f = FC ? (p1 * pq) * ia[s] : (pp.cx2[s] * (p1 * pq)) * ia[s];
        C<T> fS = f * S;
        sum = sum + fS;
        if (want_mag) {
            const T ay = cabs1(nd.y);
            T kq = ay * rcp(cabs1(ypq));
            T kk;
            if (pp.same[s]) {
                kk = kq;
            } else if (pp.full[s]) {
                const C<T> yp = KConst<T>::yp(kp);
                kk = ay * (rcp(cabs1(nd.y - yp)) + rcp(cabs1(nd.y - conj(yp))));
            } else {
                kk = ay * rcp(cabs1(nd.y + pp.m2k[s]));
            }
            const T m = FC ? cabs1(fS) * cabs1(pp.cx2[s]) : cabs1(fS);
            mag += m;
            // with y, y + M2 and a exact to one rounding (binary32 ray nodes)
            // the pole terms weigh less: what remains is the rounding of the
            // node's later operations near the pole, not the cancellation
            magk += m * (kap[s] + kq + kk) * (exact_y ? T(kMixedPoleWeight) : T(1));
        }
    }
    if (want_mag) {
        const T aj = cabs1(nd.Jt);
        const T kw = sizeof(T) == 4 ? cabs1(w[0]) * trsqrt(qmin) : T(0);
        mag = aj * mag;
        magk = aj * magk + mag * (T(1) + kw);
        ea.s1 += mag;
        ea.s2 += magk * magk;
    }
    return nd.Jt * sum;
}

// Binary64 and double-float nodes of a ray, evaluated in the frame of the ray,
// for the three kinds of term whose factors are all of the form 1/(y - y0):
// terms whose two legs share their pole (P1 = P2 = 1/(s + M2): the scalar
// bubble, and the equal-pole partial-fraction terms of the dressed
// propagator), the pair of dressed terms whose k-leg is the whole propagator
// D(y) = R+/(y - y+) + R-/(y - y-) (the sector where no pole is swept), and,
// in binary64, one term whose k-leg has a pole of its own (the complex-pair
// legs of the paper's example; on a detour only its tail ray). On the ray
// y = r e2 with r = rho^2 real, so every factor of
// node_value is r and per-pass constants; for a term with M2:
//   a = x + y + M2 = e2 (r + xi),    xi  = (x + M2)/e2,
//   y + M2         = e2 (r + eta),   eta = M2/e2,
// 1/a = g/e2 and 1/(y + M2) = h/e2 with g = 1/(r + xi), h = 1/(r + eta);
// u = y/a = r g, w = 4xy/a^2 = chi u g (chi = 4x/e2), and the lead
// (delta y - Omega (x + M2))/a - Omega1 w = (delta r - Omega xi) g - Omega1 w.
// The node's value Jt P1 (1/(y + M2)) (1/a) S is m (eD/e2^3) H h g S with
// m = rho^(D-1) W and H = h (shared pole), H = R+ h+ + R- h- (the whole
// propagator; its terms' M2 are -y+ and -y-, in that order) or
// H = 1/(r + M2k/e2) (a k-leg pole M2k of its own); eD/e2^3 joins
// the term's factor c 2x. The real reciprocals 1/|r + xi|^2 and
// 1/|r + eta|^2 (and 1/|r + M2k/e2|^2) come from one reciprocal of their
// product. No node forms y, the measure or a complex reciprocal.
// Double-float keeps binary32's range by the scale sigma = 1/(1 + r) from
// its table: it forms g' = g/sigma and h' = h/sigma from (r + xi) sigma and
// (r + eta) sigma, and takes m sigma^3, so that m H h g = (m sigma^3) H' h' g'.
template <typename T>
struct RotPre {
    C<T> xi, eta, chi, om;   // (x + M2)/e2, M2/e2, 4x/e2, Omega xi
    C<T> etak;               // distinct k-leg pole: M2k/e2
    T xi2, eta2, etak2;      // binary64: (Im xi)^2, (Im eta)^2, (Im etak)^2
};

template <typename T>
__device__ __forceinline__ RotPre<T> rot_pre(const KParams &kp, C<T> x, C<T> e2, C<T> m2,
                                             C<T> m2k)
{
    RotPre<T> rp;
    const C<T> ei = cinv(e2);
    rp.xi = (x + m2) * ei;
    rp.eta = m2 * ei;
    rp.chi = (T(4) * x) * ei;
    rp.om = T(kp.Omega) * rp.xi;
    rp.xi2 = rp.xi.i * rp.xi.i;
    rp.eta2 = rp.eta.i * rp.eta.i;
    if constexpr (std::is_same<T, double>::value) {
        rp.etak = m2k * ei;
        rp.etak2 = rp.etak.i * rp.etak.i;
    }
    return rp;
}

// Kinds of ray-frame term (node_rot): both legs on one pole, the two terms of
// the whole dressed propagator, one term whose k-leg has a pole of its own
enum { ROT_SHARED = 0, ROT_WHOLE = 1, ROT_DISTINCT = 2 };

// Two-term ray passes: each term's angular sum on its own compressed rule
// (1), or both on the larger of the two (0)
#ifndef GFC_SPLIT_RULES
#define GFC_SPLIT_RULES 1
#endif
// Ray-frame nodes for terms whose k-leg has a pole of its own (1), or the
// general node code for them (0)
#ifndef GFC_RDIST
#define GFC_RDIST 1
#endif

// Ray node k into the terms' pass sums ps (each term's factor c 2x eD/e2^3
// left out), for terms of kind MODE (ROT_*). TAIL: node k of the mapped ray
// from |q| = rho0 (the tail of a detour), else of the ray from q = 0. Returns
// the angular pairs evaluated for each term (x: the first, y: the second),
// negated when they were the full table's.
template <typename T, int NP, int NT, int MODE, bool TAIL>
__device__ __forceinline__ int2 node_rot(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                        const T *stab, const void *srules,
                                        const RotPre<T> (&rp)[NT], int k, T rho0, C<T> (&ps)[NT])
{
    constexpr bool D64 = std::is_same<T, double>::value;
    static_assert(MODE != ROT_WHOLE || NT == 2, "the whole propagator has two terms");
    static_assert(MODE != ROT_DISTINCT || NT == 1, "a distinct k-leg pole has one term");
    // rs = r sigma, sg = sigma, m = rho^(D-1) W sigma^3 (binary64: sigma = 1)
    T rs, sg, m;
    if constexpr (TAIL) {
        T rho, W;
        load2<T>(kp, 0, k, rho, W);
        rho = rho + rho0;
        const T r = rho * rho;
        const T mm = (kp.dim == 4 ? r * rho : r) * W;
        if constexpr (D64) {
            rs = r;
            m = mm;
        } else {
            sg = rcp(T(1) + r);
            rs = r * sg;
            m = ((mm * sg) * sg) * sg;
        }
    } else if constexpr (D64) {
        const double2 v = __ldg(kp.rayp64 + k);
        rs = v.x;
        m = v.y;
    } else {
        const float4 a = __ldg(kp.rayq_df + 2 * k), b = __ldg(kp.rayq_df + 2 * k + 1);
        rs = T(a.x, a.y);
        sg = T(a.z, a.w);
        m = T(b.x, b.y);
    }
    C<T> g[NT], h[NT], u[NT], w[NT], hk;
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        T t1, t2, x1, x2, n1, n2;
        if constexpr (D64) {
            t1 = rs + rp[s].xi.r;
            t2 = rs + rp[s].eta.r;
            x1 = rp[s].xi.i;
            x2 = rp[s].eta.i;
            n1 = fma(t1, t1, rp[s].xi2);
            n2 = fma(t2, t2, rp[s].eta2);
        } else {
            t1 = fma(rp[s].xi.r, sg, rs);
            t2 = fma(rp[s].eta.r, sg, rs);
            x1 = rp[s].xi.i * sg;
            x2 = rp[s].eta.i * sg;
            n1 = fma(t1, t1, x1 * x1);
            n2 = fma(t2, t2, x2 * x2);
        }
        T s1, s2;
        if constexpr (MODE == ROT_DISTINCT) {
            T t3, x3, n3;
            if constexpr (D64) {
                t3 = rs + rp[s].etak.r;
                x3 = rp[s].etak.i;
                n3 = fma(t3, t3, rp[s].etak2);
            } else {
                t3 = fma(rp[s].etak.r, sg, rs);
                x3 = rp[s].etak.i * sg;
                n3 = fma(t3, t3, x3 * x3);
            }
            const T n12 = n1 * n2;
            const T R = rcp(n12 * n3);
            const T r12 = R * n3, s3 = R * n12;
            s1 = r12 * n2;
            s2 = r12 * n1;
            hk = {t3 * s3, -(x3 * s3)};
        } else {
            const T R = rcp(n1 * n2);
            s1 = R * n2;
            s2 = R * n1;
        }
        g[s] = {t1 * s1, -(x1 * s1)};
        h[s] = {t2 * s2, -(x2 * s2)};
        u[s] = rs * g[s];
        C<T> ug;
        if constexpr (D64) ug = u[s] * g[s];
        else ug = u[s] * (sg * g[s]);
        w[s] = rp[s].chi * ug;
    }
    T A[NT], B[NT], qm;
    int2 np = {0, 0};
    if constexpr (NT == 2 && GFC_SPLIT_RULES) {
#pragma unroll
        for (int s = 0; s < NT; ++s) {
            const C<T> ws[1] = {w[s]};
            T As[1], Bs[1];
            const int n = pair_sums<T, NP, 1>(kp, tab, kp.npair, stab, srules, ws, As, Bs, qm);
            A[s] = As[0];
            B[s] = Bs[0];
            if (s == 0) np.x = n;
            else np.y = n;
        }
    } else {
        const int n = pair_sums<T, NP, NT>(kp, tab, kp.npair, stab, srules, w, A, B, qm);
        np.x = n;
        np.y = NT == 2 ? n : 0;
    }
    const T Om1 = KConst<T>::om1(kp), del = KConst<T>::del(kp);
    C<T> H = {T(0), T(0)};
    if constexpr (MODE == ROT_WHOLE) {
        const C<T> Rp = KConst<T>::Rp(kp);
        H = Rp * h[0] + conj(Rp) * h[NT - 1];
    } else if constexpr (MODE == ROT_DISTINCT) {
        H = hk;
    }
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        const C<T> T2 = {fma(-w[s].r, B[s], A[s]), w[s].i * B[s]};
        C<T> L;
        if constexpr (D64) L = C<T>{fma(del, rs, -rp[s].om.r), -rp[s].om.i} * g[s];
        else L = C<T>{fma(del, rs, -(rp[s].om.r * sg)), -(rp[s].om.i * sg)} * g[s];
        const C<T> lead = {fma(-Om1, w[s].r, L.r), fma(-Om1, w[s].i, L.i)};
        const C<T> vmw = {fma(T(4), u[s].r, -w[s].r), fma(T(4), u[s].i, -w[s].i)};
        const C<T> vw = vmw * w[s];
        const C<T> S = {fma(vw.r, T2.r, fma(-vw.i, T2.i, lead.r)),
                        fma(vw.r, T2.i, fma(vw.i, T2.r, lead.i))};
        const C<T> hh = MODE == ROT_SHARED ? h[s] * h[s] : H * h[s];
        const C<T> fS = (hh * g[s]) * S;
        ps[s].r = fma(m, fS.r, ps[s].r);
        ps[s].i = fma(m, fS.i, ps[s].i);
    }
    return np;
}

// ----------------------------------------------------------------------------
// compensated accumulation
// ----------------------------------------------------------------------------
template <typename T>
struct Acc {
    T sr, cr, si, ci;
    __device__ __forceinline__ void init() { sr = cr = si = ci = T(0); }
};

// TwoSum (Knuth) on each component: s + v = t + err exactly
template <typename T>
__device__ __forceinline__ void two_sum_add(T &s, T &c, T v)
{
    T t = s + v;
    T bp = t - s;
    T err = (s - (t - bp)) + (v - bp);
    s = t;
    c += err;
}

// binary32: compensated (TwoSum) radial sums; binary64: plain sums (at most
// n_r/32 terms per lane, error far below the FP64 tolerance); double-float:
// sums in double-float
__device__ __forceinline__ void acc_add(Acc<float> &a, C<float> v)
{
    two_sum_add(a.sr, a.cr, v.r);
    two_sum_add(a.si, a.ci, v.i);
}
__device__ __forceinline__ void acc_add(Acc<double> &a, C<double> v)
{
    a.sr += v.r;
    a.si += v.i;
}
__device__ __forceinline__ void acc_add(Acc<df> &a, C<df> v)
{
    a.sr = a.sr + v.r;
    a.si = a.si + v.i;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------------------------
// the evaluation kernel
// ----------------------------------------------------------------------------
__device__ __forceinline__ void point_x(const KParams &kp, int64_t p, double &xr, double &xi)
{
    if (kp.use_grid) {
        // re0 + (i + 1/2) dre with separate roundings (no FMA), as written
        int i = (int)(p / kp.gn), j = (int)(p - (int64_t)i * kp.gn);
        xr = __dadd_rn(kp.re0, __dmul_rn(i + 0.5, kp.dre));
        xi = __dadd_rn(kp.im0, __dmul_rn(j + 0.5, kp.dim_im));
    } else {
        xr = kp.x[2 * p];
        xi = kp.x[2 * p + 1];
    }
}

// Node groups of a point's contour (mixed precision, partial routing): the
// point's iterations -- 32 consecutive nodes of a pass, one per lane --
// numbered across its passes, gsz iterations per group, at most kMaxGroups
// groups. `mask` (0: all) selects the groups a launch evaluates; with `snap`
// set (the binary32 bulk), every group end records each lane's running
// compensated sum in snap[group][lane] and the warp's error scale of the
// group in gerr[group].
struct Groups {
    unsigned mask;
    int gsz, ngroups;
    float4 *snap;
    float2 *gerr;
};
// position of a lane's loop in the groups
struct GroupCursor {
    int g, left;   // current group; iterations left in it
};

// the warp's (sum M, sum (M kappa)^2) of the group just ended, stored by lane 0
__device__ __forceinline__ void group_end(const Groups &gr, int g, int lane, const Acc<float> &acc,
                                          ErrAcc<float> &ea)
{
    gr.snap[g * 32 + lane] = make_float4(acc.sr, acc.cr, acc.si, acc.ci);
    float s1 = ea.s1, s2 = ea.s2;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) gr.gerr[g] = make_float2(s1, s2);
    ea.s1 = ea.s2 = 0.0f;
}

// One pass of a point's contour, the lane's share of its nodes (those of
// the groups the mask selects). CL = 1 (the variant kernels) compiles in the
// options that the default kernels leave out so as to carry none of their
// registers: the closed-form angular integral and the clustered radial rule.
// Returns the nodes of the pass the warp evaluated. GM selects the group
// handling at compile time: 0 none (every node), 1 the groups of gr.mask,
// 2 every node with the binary32 bulk's group records.
template <typename T, int NP, int NTT, int CL, int GM = 0>
__device__ __forceinline__ int run_pass(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                        const T *stab, const void *srules, const Plan<T> &P,
                                        int pass, C<T> x, C<T> e2, C<T> eD, int lane, Acc<T> &acc,
                                        ErrAcc<T> &ea, T &qall, int &pairs, int &pfull,
                                        const Groups &gr, GroupCursor &cur, C<T> e2lo, C<T> xlo)
{
    const PassPre<T, NTT> pp = pass_pre<T, NTT, (GM == 2 ? 1 : 0)>(kp, P, pass, x, xlo);
    const bool ray = P.kind[pass] == PASS_RAY;
    const int nn = ray ? kp.n_r : 3 * kp.n_s + kp.n_r;
    DetourPre<T> *dps = detour_slot<T>();
    if (!ray) {
        __syncwarp();
        if (lane == 0) *dps = detour_pre<T>(kp, P.eth, P.yp, x);
        __syncwarp();
    }
    // binary32 mapped rays from q = 0 use nodes with y exact (see ray_node_exact_y)
    const bool exact_y = std::is_same<T, float>::value && ray && !(CL && P.clus);
    // one term (binary64 and double-float): the pass's factor c 2x multiplies
    // the lane's sum of the pass once instead of every node (binary32 keeps
    // it per node, where its compensated sum and error scale were set up)
    constexpr int FC = (NTT == 1 && !std::is_same<T, float>::value) ? 1 : 0;
    C<T> ps = {T(0), T(0)};
    int evaluated = 0;
    auto count = [&](int np) {
                if (np < 0) {
                    pfull -= np;
                    pairs -= np;
                } else {
                    pairs += np;
                }
    };
    auto rcount = [&](int2 np) {
        count(np.x);
        count(np.y);
    };
    // binary64 and double-float passes whose terms all share their poles,
    // carry the two terms of the whole dressed propagator, or are one term
    // with a k-leg pole of its own, without the error-scale output: ray
    // nodes in the frame of the ray (node_rot; on a detour only its tail
    // ray), each term's pass factor c 2x eD/e2^3
    constexpr bool ROT = !std::is_same<T, float>::value && !CL;
    // (distinct k-leg poles in binary64 only: in double-float their extra
    // registers would spill in the one-term kernels, held to 128)
    constexpr bool RDIST = std::is_same<T, double>::value && GFC_RDIST;
    int mode = -1;
    RotPre<T> rp[NTT];
    C<T> kpass[NTT], pr[NTT];
    T rho0 = T(0);
    if constexpr (ROT) {
        if (kp.cond_out == nullptr && pp.nt == NTT) {
            if (NTT == 1)
                mode = pp.same[0] ? ROT_SHARED : ((RDIST && !pp.full[0]) ? ROT_DISTINCT : -1);
            else if (pp.full[0] && pp.full[NTT - 1])
                mode = ROT_WHOLE;
            else if (pp.same[0] && pp.same[NTT - 1])
                mode = ROT_SHARED;
        }
        // a detour's first segments are not on the ray; its tail is
        if (!ray && mode != ROT_DISTINCT) mode = -1;
        if (mode >= 0) {
            const C<T> ei = cinv(e2);
            const C<T> f = eD * (ei * (ei * ei));
#pragma unroll
            for (int s = 0; s < NTT; ++s) {
                rp[s] = rot_pre<T>(kp, x, e2, pp.m2q[s], pp.m2k[s]);
                kpass[s] = pp.cx2[s] * f;
                pr[s] = {T(0), T(0)};
            }
            if constexpr (RDIST)
                if (!ray) rho0 = dps->sqRd;
        }
    }
    auto node = [&](int k) {
                Node<T> nd;
                if (!ray)
                    nd = detour_node<T>(kp, k, e2, eD, *dps);
                else if (CL && P.clus)
                    nd = ray_node_cl<T>(kp, k, e2, eD, P.cl_c, P.cl_d, P.cl_eta);
                else if constexpr (std::is_same<T, float>::value)
                    nd = GM == 2 ? ray_node_exact_y(kp, k, e2, eD, e2lo) : ray_node_exact_y(kp, k, e2, eD);
                else
                    nd = ray_node<T>(kp, k, e2, eD);
                T qm;
                int np;
                C<T> v = node_value<T, NP, NTT, CL, FC, (GM == 2 ? 1 : 0)>(kp, tab, stab, srules, pp,
                                                                           x, nd, ea, qm, np, exact_y);
                if constexpr (FC) ps = ps + v;
                else acc_add(acc, v);
                qall = fmin(qall, qm);
                count(np);
    };
    // node k of the pass in the frame of the ray (mode >= 0)
    auto rnode = [&](int k) {
        if constexpr (ROT) {
            if constexpr (NTT == 1) {
                if (mode == ROT_SHARED) {
                    rcount(node_rot<T, NP, NTT, ROT_SHARED, false>(kp, tab, stab, srules, rp, k, rho0, pr));
                } else if constexpr (RDIST) {
                    if (ray)
                        rcount(node_rot<T, NP, NTT, ROT_DISTINCT, false>(kp, tab, stab, srules, rp, k,
                                                                         rho0, pr));
                    else if (k < 3 * kp.n_s)
                        node(k);
                    else
                        rcount(node_rot<T, NP, NTT, ROT_DISTINCT, true>(kp, tab, stab, srules, rp,
                                                                        k - 3 * kp.n_s, rho0, pr));
                }
            } else {
                if (mode == ROT_WHOLE)
                    rcount(node_rot<T, NP, NTT, ROT_WHOLE, false>(kp, tab, stab, srules, rp, k, rho0, pr));
                else
                    rcount(node_rot<T, NP, NTT, ROT_SHARED, false>(kp, tab, stab, srules, rp, k, rho0, pr));
            }
        }
    };
    if constexpr (GM == 0) {
        if (ROT && mode >= 0) {
            if constexpr (ROT) {
                if (mode == ROT_SHARED) {
                    for (int k = lane; k < nn; k += 32)
                        rcount(node_rot<T, NP, NTT, ROT_SHARED, false>(kp, tab, stab, srules, rp, k, rho0, pr));
                } else if constexpr (RDIST || NTT == 2) {
                    for (int k = lane; k < nn; k += 32) rnode(k);
                }
            }
        } else {
            for (int k = lane; k < nn; k += 32) node(k);
        }
        evaluated = nn;
    } else {
        auto groups = [&](auto &&fn) {
            for (int base = 0; base < nn; base += 32) {
                // warp-uniform: the group of this iteration is selected
                if (GM == 2 || (cur.g < kMaxGroups && ((gr.mask >> cur.g) & 1u))) {
                    evaluated += min(32, nn - base);
                    if (base + lane < nn) fn(base + lane);
                }
                if (--cur.left == 0) {
                    if constexpr (GM == 2 && std::is_same<T, float>::value)
                        group_end(gr, cur.g, lane, acc, ea);
                    cur.left = gr.gsz;
                    ++cur.g;
                }
            }
        };
        if (ROT && mode >= 0) {
            if constexpr (RDIST || NTT == 2)
                groups(rnode);
            else if constexpr (ROT)
                groups([&](int k) {
                    rcount(node_rot<T, NP, NTT, ROT_SHARED, false>(kp, tab, stab, srules, rp, k, rho0, pr));
                });
        } else {
            groups(node);
        }
    }
    if (ROT && mode >= 0) {
        C<T> v = kpass[0] * pr[0];
#pragma unroll
        for (int s = 1; s < NTT; ++s) v = v + kpass[s] * pr[s];
        // (a detour's segments before its tail: the general nodes' sum)
        if constexpr (FC && RDIST) v = v + pp.cx2[0] * ps;
        acc_add(acc, v);
    } else if constexpr (FC) {
        acc_add(acc, pp.cx2[0] * ps);
    }
    return evaluated;
}

// Sum over one point's contour (the groups gr.mask selects), per lane, into
// acc; returns the number of contour nodes evaluated. With gr.snap set (the
// binary32 bulk with partial routing) it first sizes the groups: the fewest
// iterations per group that give at most kMaxGroups groups.
template <typename T, int NP, int NT, int CL, int GM = 0>
__device__ __forceinline__ int point_sum(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                         const T *stab, const void *srules, double xr, double xi,
                                         int lane, Acc<T> &acc, ErrAcc<T> &ea, T &qall,
                                         int &pairs, int &pfull, Groups &gr)
{
    const Plan<T> P = make_plan<T, CL>(kp, xr, xi);
    const C<T> x = cvt<T>(xr, xi);
    // e^{i D theta} of the ray, once per point
    C<T> e2 = P.eth * P.eth;
    C<T> e2lo = {T(0), T(0)}, xlo = {T(0), T(0)};
    if constexpr (GM == 2) {
        // the binary32 bulk with partial routing puts its ray nodes on the
        // exact direction x/|x| (binary32 value and remainder): the node
        // groups evaluated again in the fallback arithmetic lie on that ray,
        // and a ray turned by the direction's rounding would change the
        // kept groups' sum coherently
        const double ax = sqrt(xr * xr + xi * xi);
        const double dr = xr / ax, di = xi / ax;
        e2 = {(float)dr, (float)di};
        e2lo = {(float)(dr - (double)e2.r), (float)(di - (double)e2.i)};
        // and x itself: its remainder joins every node's a = x + y + M2 and w
        xlo = {(float)(xr - (double)x.r), (float)(xi - (double)x.i)};
        // (held in registers: not recomputed in binary64 per node)
        asm volatile("" : "+f"(e2.r), "+f"(e2.i), "+f"(e2lo.r), "+f"(e2lo.i), "+f"(xlo.r), "+f"(xlo.i));
    }
    const C<T> eD = kp.dim == 4 ? e2 * e2 : e2 * P.eth;
    if (GM == 2) {
        int iters = 0;
        for (int pass = 0; pass < P.npass; ++pass)
            iters += ((P.kind[pass] == PASS_RAY ? kp.n_r : 3 * kp.n_s + kp.n_r) + 31) / 32;
        gr.gsz = (iters + kMaxGroups - 1) / kMaxGroups;
        gr.ngroups = (iters + gr.gsz - 1) / gr.gsz;
    }
    GroupCursor cur = {0, gr.gsz};
    int total = 0;
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
        if (pass >= P.npass) break;
        if (NT > 1 && P.nterm[pass] == 2)
            total += run_pass<T, NP, (NT > 1 ? 2 : 1), CL, GM>(kp, tab, stab, srules, P, pass, x, e2,
                                                              eD, lane, acc, ea, qall, pairs, pfull,
                                                              gr, cur, e2lo, xlo);
        else
            total += run_pass<T, NP, 1, CL, GM>(kp, tab, stab, srules, P, pass, x, e2, eD, lane, acc,
                                                ea, qall, pairs, pfull, gr, cur, e2lo, xlo);
    }
    if constexpr (std::is_same<T, float>::value) {
        // the last group, if the iterations end inside it
        if (GM == 2 && cur.left != gr.gsz) group_end(gr, cur.g, lane, acc, ea);
    }
    return total;
}

__device__ __forceinline__ void list_append(const KParams &kp, int64_t p)
{
    unsigned long long k = atomicAdd(kp.list_count, 1ULL);
    kp.list[k] = p;
}

// compensated binary32 pairs (hi, lo) summed over the warp, TwoSum on the
// high parts; every lane receives the sum
__device__ __forceinline__ void warp_pair_sum(float &hr, float &lr, float &hi, float &li)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ohr = __shfl_xor_sync(0xffffffffu, hr, o), olr = __shfl_xor_sync(0xffffffffu, lr, o);
        float ohi = __shfl_xor_sync(0xffffffffu, hi, o), oli = __shfl_xor_sync(0xffffffffu, li, o);
        float cr = 0.0f, ci = 0.0f;
        two_sum_add(hr, cr, ohr);
        two_sum_add(hi, ci, ohi);
        lr = lr + olr + cr;
        li = li + oli + ci;
    }
}

// A warp's per-group error scales of the binary32 bulk (shared memory, one
// slot per warp of a block of 256)
__device__ __forceinline__ float2 *group_err_slot()
{
    __shared__ float2 slots[8][kMaxGroups];
    return slots[threadIdx.x >> 5];
}

// Epilogue of the binary32 bulk with partial routing. The point's rounding
// error estimate is the one of the plain bulk (kMixedErrFactor 2^-24 E, E =
// K_D (sqrt(sum (M kappa)^2) + sum M) over its nodes). A point that passes
// keeps its binary32 value. A point next to a pinch goes whole to the
// binary64 list. Otherwise the node groups with the largest share of E
// (S1_g + sqrt(S2_g), S1_g = sum M and S2_g = sum (M kappa)^2 over group g)
// are taken out one by one until the rest passes; the bulk writes the
// compensated binary32 sum of the kept groups (each lane's running sum less
// the removed groups' parts, from its snapshots at the group ends), and the
// point goes to the node list with the mask of the removed groups, whose
// nodes the fallback kernel evaluates and adds.
__device__ __forceinline__ void bulk_partial_epilogue(const KParams &kp, int64_t p, int lane,
                                                      const Acc<float> &acc, float qall,
                                                      const Groups &gr, double *out)
{
    __syncwarp();
    const float2 ge = lane < gr.ngroups ? gr.gerr[lane] : make_float2(0.0f, 0.0f);
    float s1 = ge.x, s2 = ge.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    float hr = acc.sr, lr = acc.cr, hi = acc.si, li = acc.ci;
    warp_pair_sum(hr, lr, hi, li);
    float qpt = qall;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qpt = fminf(qpt, __shfl_xor_sync(0xffffffffu, qpt, o));
    const double gr0 = kp.K_D * ((double)hr + (double)lr) - kp.g0mu[0];
    const double gi0 = kp.K_D * ((double)hi + (double)li) - kp.g0mu[1];
    // the largest sqrt(sum (M kappa)^2) + sum M that passes
    const float lim = (float)(kp.mixed_rtol * sqrt(gr0 * gr0 + gi0 * gi0) /
                              (kMixedErrFactor * 5.9604644775390625e-8 * kp.K_D));
    if (!(kp.mixed_rtol > 0.0) || (sqrtf(s2) + s1 <= lim && !(qpt < kMixedPinchQ))) {
        if (lane == 0) {
            out[0] = gr0;
            out[1] = gi0;
            if (kp.cond_out) kp.cond_out[p] = kp.K_D * ((double)sqrtf(s2) + (double)s1);
        }
        __syncwarp();
        return;
    }
    if (qpt < kMixedPinchQ || !(sqrtf(s2) + s1 <= lim * (float)kPartialMax)) {
        // next to a pinch, or where the estimate fails by more than
        // kPartialMax (the badly conditioned points next to the negative
        // real axis, whose kept groups the estimate does not bound), no
        // binary32 part is kept: every group goes to the fallback, which adds
        // the whole sum to -G0(mu2)
        if (lane == 0) {
            out[0] = -kp.g0mu[0];
            out[1] = -kp.g0mu[1];
            if (kp.cond_out) kp.cond_out[p] = 0.0;
            const unsigned long long k = atomicAdd(kp.node_list_count, 1ULL);
            kp.node_list[k] = NodeEntry{p, gr.ngroups >= 32 ? 0xffffffffu : (1u << gr.ngroups) - 1u, gr.gsz};
        }
        __syncwarp();
        return;
    }
    // take out the groups with the largest share, one per round (the same
    // decision on every lane: the sums above are butterflies), until the rest
    // passes with the margin kPartialMargin
    const float S1 = ge.x, S2 = ge.y;
    float score = lane < gr.ngroups ? S1 + sqrtf(S2) : -1.0f;
    float r1 = s1, r2 = s2;
    unsigned mask = 0u;
    const float limk = lim * (float)(1.0 / kPartialMargin);
    while (!(sqrtf(fmaxf(r2, 0.0f)) + fmaxf(r1, 0.0f) <= limk)) {
        // non-negative binary32 values order as their bit patterns
        const unsigned key = score >= 0.0f ? __float_as_uint(score) + 1u : 0u;
        const unsigned mx = __reduce_max_sync(0xffffffffu, key);
        if (mx == 0u) break;                       // every group is out
        const int g = __ffs(__ballot_sync(0xffffffffu, key == mx)) - 1;
        mask |= 1u << g;
        r1 -= __shfl_sync(0xffffffffu, S1, g);
        r2 -= __shfl_sync(0xffffffffu, S2, g);
        if (lane == g) score = -1.0f;
    }
    // the lane's kept sum: its total less each removed group's part, the
    // difference of its snapshots at the group's end and at the one before
    float kr = acc.sr, klr = acc.cr, ki = acc.si, kli = acc.ci;
    for (unsigned m = mask; m; m &= m - 1u) {
        const int g = __ffs(m) - 1;
        const float4 a = gr.snap[g * 32 + lane];
        const float4 b = g > 0 ? gr.snap[(g - 1) * 32 + lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        two_sum_add(kr, klr, -a.x);
        two_sum_add(kr, klr, b.x);
        klr += b.y - a.y;
        two_sum_add(ki, kli, -a.z);
        two_sum_add(ki, kli, b.z);
        kli += b.w - a.w;
    }
    warp_pair_sum(kr, klr, ki, kli);
    if (lane == 0) {
        out[0] = kp.K_D * ((double)kr + (double)klr) - kp.g0mu[0];
        out[1] = kp.K_D * ((double)ki + (double)kli) - kp.g0mu[1];
        // the error scale of the part kept in binary32
        if (kp.cond_out)
            kp.cond_out[p] = kp.K_D * ((double)sqrtf(fmaxf(r2, 0.0f)) + (double)fmaxf(r1, 0.0f));
        const unsigned long long k = atomicAdd(kp.node_list_count, 1ULL);
        kp.node_list[k] = NodeEntry{p, mask, gr.gsz};
    }
    __syncwarp();
}

// Evaluates point p of the request described by kp under `mode`; the whole
// warp calls it with the same p. Under MODE_NODES only the node groups in
// gmask (gsz iterations each) are evaluated and added to G. GM: the group
// handling of run_pass, fixed per call site (1 for MODE_NODES, 2 for the
// binary32 bulk with partial routing, else 0).
template <typename T, int NP, int NT, int CL, int GM = 0>
__device__ __forceinline__ void eval_point(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                           const T *stab, const void *srules, int64_t p, int mode,
                                           int lane, unsigned gmask = 0u, int gsz = 1)
{
    double xr, xi;
    point_x(kp, p, xr, xi);
    double *out = kp.G + 2 * p;
    if (xi == 0.0 && (xr < 0.0 || xr == kp.mu2)) {
        // the cut side of the real axis is undefined (NaN); G(mu2) = 0 by
        // the subtraction
        if ((mode == MODE_ALL || mode == MODE_BULK32) && lane == 0) {
            double v = xr < 0.0 ? __longlong_as_double(0x7ff8000000000000ULL) : 0.0;
            out[0] = v;
            out[1] = v;
            if (kp.cond_out) kp.cond_out[p] = 0.0;
        }
        return;
    }
    if (mode == MODE_BULK32 && in_band(kp, xr, xi)) {
        if (lane == 0) list_append(kp, p);
        return;
    }
    Groups gr = {gmask, gsz, 0, nullptr, nullptr};
    if constexpr (GM == 2) {
        // partial routing: this warp's snapshot slot and group table (the
        // caller checked the slot against kp.snap_slots)
        const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
        gr.snap = kp.snap + slot * (kMaxGroups * 32);
        gr.gerr = group_err_slot();
    }
    Acc<T> acc;
    acc.init();
    ErrAcc<T> ea = {T(0), T(0)};
    T qall = T(1e30);
    int pairs = 0, pfull = 0;
    int nodes = point_sum<T, NP, NT, CL, GM>(kp, tab, stab, srules, xr, xi, lane, acc, ea, qall,
                                             pairs, pfull, gr);
    if (kp.node_count && lane == 0)
        atomicAdd(kp.node_count, (unsigned long long)nodes * (unsigned long long)(2 * kp.npair));
    if (kp.pair_count) {
        unsigned long long pw = (unsigned long long)pairs, pf = (unsigned long long)pfull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pw += __shfl_xor_sync(0xffffffffu, pw, o);
            pf += __shfl_xor_sync(0xffffffffu, pf, o);
        }
        if (lane == 0) {
            atomicAdd(kp.pair_count, pw);
            if (kp.pair_full_count) atomicAdd(kp.pair_full_count, pf);
        }
    }
    if constexpr (GM == 2) {
        bulk_partial_epilogue(kp, p, lane, acc, (float)qall, gr, out);
        return;
    }
    double sr, si, cond;
    if constexpr (std::is_same<T, float>::value) {
        // binary32 throughout (the FP64 pipe is 1/64 of the binary32 one): the
        // lanes' compensated sums (hi, lo) are reduced as pairs, TwoSum on the
        // high parts; the error scale needs no more than binary32
        float hr = acc.sr, lr = acc.cr, hi = acc.si, li = acc.ci, s1 = ea.s1, s2 = ea.s2;
        warp_pair_sum(hr, lr, hi, li);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        sr = (double)hr + (double)lr;
        si = (double)hi + (double)li;
        cond = kp.K_D * ((double)sqrtf(s2) + (double)s1);
    } else {
        sr = warp_sum((double)acc.sr + (double)acc.cr);
        si = warp_sum((double)acc.si + (double)acc.ci);
        cond = kp.K_D * (sqrt(warp_sum((double)ea.s2)) + warp_sum((double)ea.s1));
    }
    if (mode == MODE_NODES) {
        // the removed groups' part, added to what the bulk wrote
        if (lane == 0) {
            out[0] += kp.K_D * sr;
            out[1] += kp.K_D * si;
        }
        return;
    }
    float qpt = (float)qall;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qpt = fminf(qpt, __shfl_xor_sync(0xffffffffu, qpt, o));
    if (lane == 0) {
        double gr0 = kp.K_D * sr - kp.g0mu[0], gi0 = kp.K_D * si - kp.g0mu[1];
        out[0] = gr0;
        out[1] = gi0;
        if (kp.cond_out) kp.cond_out[p] = cond;
        if (mode == MODE_BULK32 && kp.mixed_rtol > 0.0) {
            // rounding error of the binary32 sum: a small multiple of 2^-24
            // times the error scale (see ErrAcc). Next to a pinch (some node
            // with |1 - w t| < 3e-3) the discrete sum is so sensitive to the
            // binary32 rounding of x and of the nodes that no such bound
            // holds; those points go to binary64 too.
            double est = kMixedErrFactor * 5.9604644775390625e-8 * cond;
            if (!(est <= kp.mixed_rtol * sqrt(gr0 * gr0 + gi0 * gi0)) || qpt < kMixedPinchQ)
                list_append(kp, p);
        }
    }
}

template <typename T>
__device__ __forceinline__ const void *rules_of(const KParams &kp);
template <>
__device__ __forceinline__ const void *rules_of<double>(const KParams &kp) { return kp.rules64; }
template <>
__device__ __forceinline__ const void *rules_of<float>(const KParams &kp) { return kp.rules32; }
template <>
__device__ __forceinline__ const void *rules_of<df>(const KParams &kp) { return kp.rules_df; }

template <typename T>
__host__ __device__ constexpr int rule_bytes() { return sizeof(T) == 8 ? 24 : 16; }   // double, df: 3 x 8

// bytes of shared memory: the full pair table (generic kernels only), 16-byte
// aligned, then the compressed rules
template <typename T, int NP>
__host__ __device__ inline size_t smem_bytes(int npair, int rules_total)
{
    size_t a = NP > 0 ? 0 : ((sizeof(T) * 3 * npair + 15) / 16) * 16;
    return a + (size_t)rule_bytes<T>() * rules_total;
}

// Copies the pair table (NP = 0) and the compressed rules of kp to shared
// memory; every request of one launch shares them.
template <typename T, int NP>
__device__ __forceinline__ void stage_tables(const KParams &kp, const T *gtab, int npair,
                                             const T *&stab, const void *&srules)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *st = reinterpret_cast<T *>(smem_raw);
    size_t a = NP > 0 ? 0 : ((sizeof(T) * 3 * npair + 15) / 16) * 16;
    if (NP == 0)
        for (int i = threadIdx.x; i < 3 * npair; i += blockDim.x) st[i] = gtab[i];
    const int nw = rule_bytes<T>() * kp.rules_total / 4;
    const unsigned *src = reinterpret_cast<const unsigned *>(rules_of<T>(kp));
    unsigned *dst = reinterpret_cast<unsigned *>(smem_raw + a);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    stab = st;
    srules = smem_raw + a;
}

// One request: warps take points from an atomic counter until none is left.
// GMK selects the launch's kind at compile time, so that each instantiation
// carries only its own registers: 0 every point of MODE_ALL, MODE_LIST64 or
// the binary32 bulk without partial routing; 1 MODE_NODES (the node groups of
// the partially routed points); 2 the binary32 bulk with partial routing.
template <typename T, int NP, int NT, int CL, int GMK>
__device__ __forceinline__ void eval_loop(const KParams &kp, const AngTab<T, tab_size<NP>()> &tab,
                                          const T *gtab)
{
    const T *stab;
    const void *srules;
    stage_tables<T, NP>(kp, gtab, kp.npair, stab, srules);
    const int lane = threadIdx.x & 31;
    // a warp without a snapshot slot evaluates its points in the plain bulk
    // (the launcher sizes the slots for every warp the grid can hold)
    const bool slot_ok =
        (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) < kp.snap_slots;
    const unsigned long long n = kp.mode == MODE_LIST64  ? *kp.list_count
                                 : kp.mode == MODE_NODES ? *kp.node_list_count
                                                         : (unsigned long long)kp.npts;
    for (;;) {
        unsigned long long p = 0;
        if (lane == 0) p = atomicAdd(kp.counter, 1ULL);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= n) break;
        if constexpr (GMK == 1) {
            const NodeEntry en = kp.node_list[p];
            eval_point<T, NP, NT, CL, 1>(kp, tab, stab, srules, en.point, MODE_NODES, lane,
                                         en.mask, en.gsz);
        } else if constexpr (GMK == 2) {
            if (slot_ok)
                eval_point<T, NP, NT, CL, 2>(kp, tab, stab, srules, (int64_t)p, MODE_BULK32, lane);
            else
                eval_point<T, NP, NT, CL, 0>(kp, tab, stab, srules, (int64_t)p, MODE_BULK32, lane);
        } else {
            int64_t pt = kp.mode == MODE_LIST64 ? kp.list[p] : (int64_t)p;
            eval_point<T, NP, NT, CL>(kp, tab, stab, srules, pt, kp.mode, lane);
        }
    }
}

// the default one-term double-float kernels held to GFC_DF_MINB blocks of 256
// threads per SM (2: 128 registers; measured on GB300, production bubble grid:
// 8.31 Mpoints/s, against 6.70 at 160 registers and one block). The binary64
// kernels are left at one block (157 registers: 1.60 Mpoints/s, against 1.57
// held to two blocks with spills).
#ifndef GFC_DF_MINB
#define GFC_DF_MINB 2
#endif
template <typename T, int NP, int NT, int CL, int GMK = 0>
__global__ void __launch_bounds__(256, (std::is_same<T, df>::value && NT == 1 && !CL) ? GFC_DF_MINB : 1)
eval_kernel(const __grid_constant__ KParams kp,
            const __grid_constant__ AngTab<T, tab_size<NP>()> tab, const T *__restrict__ gtab)
{
    eval_loop<T, NP, NT, CL, GMK>(kp, tab, gtab);
}

// the binary32 bulk with partial routing, held to the occupancy of the
// plain bulk: 3 blocks of 256 threads per SM (2 for the variant kernels)
template <typename T, int NP, int NT, int CL>
__global__ void __launch_bounds__(256, CL ? 2 : 3)
eval_bulk_partial_kernel(const __grid_constant__ KParams kp,
                         const __grid_constant__ AngTab<T, tab_size<NP>()> tab,
                         const T *__restrict__ gtab)
{
    eval_loop<T, NP, NT, CL, 2>(kp, tab, gtab);
}

// Many requests in one persistent launch (continuous batching): item i covers
// points [items[i].p0, items[i].p1) of request slot items[i].slot; offs[i] is
// its first index in the launch-wide point count. All requests of a launch
// share the angular rule (n_angular, D) held in the constant bank.
// (binary32: 3 blocks of 256 threads per SM for one term, 2 for two; the
// others one, which gives the binary64 kernel the registers it needs without
// spills)
template <typename T, int NP, int NT, int CL>
__global__ void __launch_bounds__(256, std::is_same<T, float>::value ? (NT == 1 ? 3 : 2) : 1)
eval_batch_kernel(const KParams *__restrict__ slots, const BatchItem *__restrict__ items,
                  const int64_t *__restrict__ offs, int nitems, int64_t total,
                  unsigned long long *counter, int mode,
                  const __grid_constant__ AngTab<T, tab_size<NP>()> tab, const T *__restrict__ gtab,
                  int npair)
{
    const T *stab;
    const void *srules;
    stage_tables<T, NP>(slots[items[0].slot], gtab, npair, stab, srules);
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long p = 0;
        if (lane == 0) p = atomicAdd(counter, 1ULL);
        p = __shfl_sync(0xffffffffu, p, 0);
        if (p >= (unsigned long long)total) break;
        int lo = 0, hi = nitems - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= (int64_t)p) lo = mid;
            else hi = mid - 1;
        }
        const BatchItem it = items[lo];
        const KParams &kp = slots[it.slot];
        int64_t q = it.p0 + ((int64_t)p - offs[lo]);
        eval_point<T, NP, NT, CL>(kp, tab, stab, srules, mode == MODE_LIST64 ? kp.list[q] : q,
                                  mode, lane);
    }
}

// ----------------------------------------------------------------------------
// host launchers
// ----------------------------------------------------------------------------
// SM count of the current device, cached per device (devices may differ)
static inline int sm_count()
{
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }
    if (cached[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 1;
    }
    return cached[dev];
}

template <typename T, int NP>
static void fill_tab(AngTab<T, NP> &tab, const DevTables &tb, int npair)
{
    for (int j = 0; j < NP; ++j) {
        tab.t[j] = j < npair ? T(tb.t[j]) : T(0);
        tab.e[j] = j < npair ? T(tb.e[j]) : T(0);
        tab.g[j] = j < npair ? T(tb.g[j]) : T(0);
    }
}

template <typename T>
const T *gtab_of(const DevTables &tb);
template <>
inline const double *gtab_of<double>(const DevTables &tb) { return tb.ang64; }
template <>
inline const float *gtab_of<float>(const DevTables &tb) { return tb.ang32; }
template <>
inline const df *gtab_of<df>(const DevTables &tb) { return reinterpret_cast<const df *>(tb.ang_df); }

template <typename T, int NP, int NT, int CL, int GMK = 0>
static cudaError_t run_eval(const KParams &kp, const DevTables &tb, cudaStream_t st)
{
    AngTab<T, tab_size<NP>()> tab;
    fill_tab(tab, tb, NP > 0 ? kp.npair : 0);
    size_t smem = smem_bytes<T, NP>(kp.npair, kp.rules_total);
    const void *fn;
    if constexpr (GMK == 2) fn = (const void *)eval_bulk_partial_kernel<T, NP, NT, CL>;
    else fn = (const void *)eval_kernel<T, NP, NT, CL, GMK>;
    int blocks_per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, 256, smem);
    if (err != cudaSuccess) return err;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    int64_t blocks = (kp.npts + 7) / 8;
    int64_t cap = (int64_t)sm_count() * blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if constexpr (GMK == 2)
        eval_bulk_partial_kernel<T, NP, NT, CL><<<(unsigned)blocks, 256, smem, st>>>(kp, tab,
                                                                                    gtab_of<T>(tb));
    else
        eval_kernel<T, NP, NT, CL, GMK><<<(unsigned)blocks, 256, smem, st>>>(kp, tab, gtab_of<T>(tb));
    return cudaGetLastError();
}

template <typename T, int NP, int NT, int CL>
static cudaError_t run_batch(const BatchLaunch &bl, const DevTables &tb, cudaStream_t st)
{
    AngTab<T, tab_size<NP>()> tab;
    fill_tab(tab, tb, NP > 0 ? bl.npair : 0);
    size_t smem = smem_bytes<T, NP>(bl.npair, bl.rules_total);
    int blocks_per_sm = 0;
    cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &blocks_per_sm, (const void *)eval_batch_kernel<T, NP, NT, CL>, 256, smem);
    if (err != cudaSuccess) return err;
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    int64_t blocks = (bl.total + 7) / 8;
    int64_t cap = (int64_t)sm_count() * blocks_per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    eval_batch_kernel<T, NP, NT, CL><<<(unsigned)blocks, 256, smem, st>>>(
        bl.slots, bl.items, bl.offs, bl.nitems, bl.total, bl.counter, bl.mode, tab,
        gtab_of<T>(tb), bl.npair);
    return cudaGetLastError();
}

// One launch of the evaluation kernel (one request) or of the batched kernel
// (many requests), binary arithmetic T, pair table unrolled for NP pairs (0:
// generic loop). Defined in gfc_eval_inst.cu, one object file per (T, NP).
template <typename T, int NP>
cudaError_t eval_inst(const KParams &kp, const DevTables &tb, cudaStream_t st);
template <typename T, int NP>
cudaError_t batch_inst(const BatchLaunch &bl, const DevTables &tb, bool two_terms, cudaStream_t st);

}  // namespace gfc
