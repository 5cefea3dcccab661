// gfc_eval_points_noalloc: the binary64 evaluation of gfc_eval_points for
// callers that cannot allocate device memory -- for example code that runs
// while another component owns the whole device heap (a framework's caching
// allocator, or an embedding with a fixed device-memory plan), or code that
// must not pay for the device-wide synchronisation that cudaFree (and often
// cudaMalloc) implies. Its node tables and scratch live in one file-scope
// device array of fixed size (kNoAllocBytes), so the call allocates nothing:
// no cudaMalloc, no cudaFree, no allocating library call.
//
// The tables are built on the host into static arrays of this file and
// uploaded with cudaMemcpyAsync from that pageable memory; such a copy may
// wait for the work already queued on the stream before it returns. A mutex
// serialises the calls of all host threads while the arrays are refilled.
// The device array is shared by every call in the process on a given device
// and keeps the contents of the last call; calls that overlap on the GPU (on
// different streams, or from different host threads) race on it. The first
// call on a device looks up the array's device address (cudaGetSymbolAddress)
// with that device current; make that first call before any stream capture.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "gfc.h"
#include "gfc_internal.h"

namespace gfc {

namespace {

// limits of the variant
constexpr int kNaMaxRadial = 4096;
constexpr int kNaMaxAngular = 512;
constexpr int kNaMaxG0Warps = 128;

// layout of the scratch array (bytes, each block 256-byte aligned)
constexpr size_t align256(size_t n) { return (n + 255) / 256 * 256; }
constexpr size_t kOffRad = 0;
constexpr size_t kOffRayp = kOffRad + align256(sizeof(double2) * kNaMaxRadial);
constexpr size_t kOffSeg = kOffRayp + align256(sizeof(double2) * kNaMaxRadial);
constexpr size_t kOffArc = kOffSeg + align256(sizeof(double2) * (kNaMaxRadial / 4));
constexpr size_t kOffAng = kOffArc + align256(sizeof(double2) * (kNaMaxRadial / 4));
constexpr size_t kOffPart = kOffAng + align256(sizeof(double) * 3 * (kNaMaxAngular / 2));
constexpr size_t kOffG0 = kOffPart + align256(sizeof(double) * 2 * kNaMaxG0Warps);
constexpr size_t kOffCnt = kOffG0 + align256(sizeof(double) * 2);
constexpr size_t kOffTicket = kOffCnt + align256(sizeof(unsigned long long) * kCounters);
constexpr size_t kNoAllocBytes = kOffTicket + align256(sizeof(unsigned));

}  // namespace

// The scratch of gfc_eval_points_noalloc (about 170 KB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

std::mutex g_na_mu;
unsigned char *g_na_ptr[64];     // device address of the array, per device
bool g_na_ready[64];

// host staging of the tables (static: nothing allocated per call)
double2 h_rad[kNaMaxRadial], h_rayp[kNaMaxRadial], h_seg[kNaMaxRadial / 4], h_arc[kNaMaxRadial / 4];
double h_ang[3 * (kNaMaxAngular / 2)];
double h_t[kNaMaxAngular / 2], h_e[kNaMaxAngular / 2], h_g[kNaMaxAngular / 2];
double h_gx[kNaMaxRadial], h_gw[kNaMaxRadial];

// Gauss-Legendre on [-1, 1] into caller arrays: Newton on P_n(cos theta) in
// the angle (as the table builder of the allocating path does).
void gl_into(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double th = pi * (i + 0.75) / (n + 0.5);
        for (int it = 0; it < 60; ++it) {
            double c = std::cos(th), s = std::sin(th);
            double p0 = 1.0, p1 = c;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2 * k - 1) * c * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            double q = n * (p0 - c * p1);
            double step = p1 / (-q / s);
            th -= step;
            if (std::fabs(step) < 1e-17) break;
        }
        double c = std::cos(th), s = std::sin(th);
        double p0 = 1.0, p1 = c;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2 * k - 1) * c * p1 - (k - 1) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        double d = n * (p0 - c * p1) / s;
        x[n - 1 - i] = c;
        w[n - 1 - i] = 2.0 / (d * d);
        x[i] = -c;
        w[i] = 2.0 / (d * d);
    }
    if (n % 2 == 1) x[n / 2] = 0.0;
}

}  // namespace

}  // namespace gfc

using namespace gfc;

extern "C" int gfc_eval_points_noalloc(const gfc_propagator *prop, const gfc_params *params,
                                       const double *x, int64_t npts, double *G, void *stream)
{
    int rc = check_params_c(params);
    if (rc) return rc;
    if (params->precision != GFC_FP64)
        return fail(GFC_EINVAL, "gfc_eval_points_noalloc evaluates in GFC_FP64 only");
    if (params->n_radial > kNaMaxRadial || params->n_angular > kNaMaxAngular)
        return fail(GFC_EINVAL, "gfc_eval_points_noalloc: n_radial <= 4096 and n_angular <= 512");
    if (params->n_angular % 2 || params->angular_rule != GFC_ANG_GAUSS_LEGENDRE ||
        params->radial_rule != GFC_RAD_MAPPED)
        return fail(GFC_EINVAL, "gfc_eval_points_noalloc: even n_angular, the Gauss-Legendre "
                                "angular and the mapped radial rule only");
    if (npts < 0) return fail(GFC_EINVAL, "npts < 0");
    if (npts > 0 && (!x || !G)) return fail(GFC_EINVAL, "x and G must be device pointers");
    if (((uintptr_t)x | (uintptr_t)G) & 15) return fail(GFC_EINVAL, "x and G must be 16-byte aligned");
    PropConst pc;
    if ((rc = make_prop_c(prop, params, pc))) return rc;
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(GFC_EINVAL, "device index above 63");
    cudaStream_t st = (cudaStream_t)stream;

    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ready[dev]) {
        // host code cannot use the array's name as an address: ask the runtime
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
        g_na_ptr[dev] = (unsigned char *)ptr;
        g_na_ready[dev] = true;
    }
    unsigned char *base = g_na_ptr[dev];

    // tables, as the allocating path builds them (full angular rule only)
    const double pi = 3.14159265358979323846;
    const int nr = params->n_radial, ns = nr / 4, na = params->n_angular, np = na / 2;
    const double L = params->radial_scale;
    gl_into(nr, h_gx, h_gw);
    for (int k = 0; k < nr; ++k) {
        double t = 0.5 * (h_gx[k] + 1.0), omt = 0.5 * (1.0 - h_gx[k]);
        h_rad[k] = make_double2(L * t / omt, L / (omt * omt) * 0.5 * h_gw[k]);
        // (rho^2, rho^(D-1) W) of the binary64 ray nodes
        const double r2 = h_rad[k].x * h_rad[k].x;
        h_rayp[k] = make_double2(r2, (params->dim == 4 ? r2 * h_rad[k].x : r2) * h_rad[k].y);
    }
    gl_into(ns, h_gx, h_gw);
    for (int k = 0; k < ns; ++k) {
        double t = 0.5 * (h_gx[k] + 1.0);
        h_seg[k] = make_double2(t, 0.5 * h_gw[k]);
        h_arc[k] = make_double2(std::cos(pi * t), std::sin(pi * t));
    }
    gl_into(na, h_gx, h_gw);
    double Om = 0, Om1 = 0, c_om = 0, c_om1 = 0;
    for (int j = 0; j < np; ++j) {
        double psi = 0.5 * pi * (h_gx[j] + 1.0);
        double sn = std::sin(psi), cs = std::cos(psi);
        double w = 0.5 * pi * h_gw[j] * (params->dim == 4 ? sn * sn : sn);
        double t = cs * cs;
        h_t[j] = t;
        h_e[j] = w * t * t;
        h_g[j] = w * t * t * t;
        h_ang[3 * j] = h_t[j];
        h_ang[3 * j + 1] = h_e[j];
        h_ang[3 * j + 2] = h_g[j];
        double y = w - c_om, s = Om + y;
        c_om = (s - Om) - y;
        Om = s;
        y = w * t - c_om1;
        s = Om1 + y;
        c_om1 = (s - Om1) - y;
        Om1 = s;
    }
    // copies from pageable host memory return once the source has been read,
    // so the static staging arrays can be refilled by the next call
    if ((e = cudaMemcpyAsync(base + kOffRad, h_rad, sizeof(double2) * nr, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + kOffRayp, h_rayp, sizeof(double2) * nr, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + kOffSeg, h_seg, sizeof(double2) * ns, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + kOffArc, h_arc, sizeof(double2) * ns, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(base + kOffAng, h_ang, sizeof(double) * 3 * np, cudaMemcpyHostToDevice, st)))
        return cuda_fail(e, "cudaMemcpyAsync(tables into the scratch array)");
    // the G0(mu2) reduction ticket must start at zero
    if ((e = cudaMemsetAsync(base + kOffTicket, 0, sizeof(unsigned), st)))
        return cuda_fail(e, "cudaMemsetAsync(ticket)");

    KParams kp;
    std::memset(&kp, 0, sizeof kp);
    kp.dim = params->dim;
    kp.n_r = nr;
    kp.n_s = ns;
    kp.npair = np;
    kp.rad64 = reinterpret_cast<const double2 *>(base + kOffRad);
    kp.rayp64 = reinterpret_cast<const double2 *>(base + kOffRayp);
    kp.seg64 = reinterpret_cast<const double2 *>(base + kOffSeg);
    kp.arc64 = reinterpret_cast<const double2 *>(base + kOffArc);
    kp.L = L;
    kp.r_detour = params->detour_radius;
    kp.K_D = params->dim == 4 ? 4.0 * pi / std::pow(2.0 * pi, 4) : 2.0 * pi / std::pow(2.0 * pi, 3);
    kp.mu2 = params->mu2;
    kp.Omega = Om;
    kp.Omega1 = Om1;
    kp.delta = 4.0 * Om1 - Om;
    kp.nrule = 0;               // full angular rule
    kp.rules_total = 0;
    kp.pc = pc;
    kp.cut_band = params->cut_band;
    kp.pinch_angle = params->pinch_angle;
    kp.mode = MODE_ALL;
    kp.use_grid = 0;
    kp.npts = npts;
    kp.x = x;
    kp.G = G;
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(base + kOffCnt);
    kp.g0mu = reinterpret_cast<const double *>(base + kOffG0);
    kp.counter = cnt;

    DevTables tb;
    tb.ang64 = reinterpret_cast<const double *>(base + kOffAng);
    tb.ang32 = nullptr;
    tb.t = h_t;
    tb.e = h_e;
    tb.g = h_g;
    int nw = (nr + 31) / 32;
    if (nw > kNaMaxG0Warps) nw = kNaMaxG0Warps;
    e = launch_g0mu(kp, tb, params->mu2, reinterpret_cast<double *>(base + kOffPart), nw,
                    reinterpret_cast<unsigned *>(base + kOffTicket),
                    reinterpret_cast<double *>(base + kOffG0), cnt, st);
    if (e != cudaSuccess) return cuda_fail(e, "g0mu launch");
    if (npts > 0) {
        e = launch_eval(kp, tb, ARITH_F64, st);
        if (e != cudaSuccess) return cuda_fail(e, "eval launch");
    }
    return GFC_OK;
}
