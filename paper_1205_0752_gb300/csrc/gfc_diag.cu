// Diagnostics of Step 3 (Sect. 5, Figs. 1-2): the angular integral B(x, y)
// of the (p-k) leg on a set of complex y at one x (Fig. 1's density plot,
// whose discontinuities trace the branch cut of eq. 25), and the map of the
// x for which that cut leaves the positive real y-axis free (region 1 of
// Fig. 2, where the original contour can be kept).
#include <cmath>
#include <complex>
#include <cstring>

#include "gfc_kernels.cuh"

namespace gfc {

namespace {

// P2(s) = sum_t c_t/(s + M_t), the (p-k) leg as given (no relabelling)
struct LegTerms {
    int n;
    double c_re[2], c_im[2], m_re[2], m_im[2];
};

int leg_terms(const gfc_propagator *g, LegTerms &L)
{
    std::memset(&L, 0, sizeof L);
    if (g->kind == GFC_PROP_SCALAR) {
        L.n = 1;
        L.c_re[0] = 1.0;
        L.m_re[0] = g->m2;
    } else if (g->kind == GFC_PROP_CPAIR) {
        L.n = 1;
        L.c_re[0] = 1.0;
        L.m_re[0] = g->mq2_re;
        L.m_im[0] = g->mq2_im;
    } else if (g->kind == GFC_PROP_DRESSED) {
        // (s + a)/(s^2 + b s + c) = R+/(s - y+) + R-/(s - y-)
        std::complex<double> yp(-0.5 * g->b, 0.5 * std::sqrt(4 * g->c - g->b * g->b));
        std::complex<double> ym = std::conj(yp);
        std::complex<double> Rp = (yp + g->a) / (yp - ym), Rm = (ym + g->a) / (ym - yp);
        L.n = 2;
        L.c_re[0] = Rp.real(); L.c_im[0] = Rp.imag(); L.m_re[0] = -yp.real(); L.m_im[0] = -yp.imag();
        L.c_re[1] = Rm.real(); L.c_im[1] = Rm.imag(); L.m_re[1] = -ym.real(); L.m_im[1] = -ym.imag();
    } else {
        return fail(GFC_EINVAL, "unknown propagator kind");
    }
    return GFC_OK;
}

// B(x, y) = sum_t c_t int sin^(D-2) psi [1/(s + M_t) - 1/(y + M_t)] dpsi. Per
// pole, pairing psi with pi - psi gives (y - s)/(s + M) -> (2x/a) (v t - 1)/
// (1 - w t), a = x + y + M, v = 4y/a, w = 4xy/a^2, t = cos^2 psi: the same
// paired sum S as the evaluation kernels, here over the full pair table (or
// in closed form), divided by (y + M).
__global__ void __launch_bounds__(256)
angular_map_kernel(const __grid_constant__ KParams kp, const double *__restrict__ ang,
                   LegTerms L, double xr, double xi, const double *__restrict__ y, int64_t ny,
                   double *__restrict__ B)
{
    const C<double> x = {xr, xi};
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < ny;
         p += (int64_t)gridDim.x * blockDim.x) {
        const C<double> yy = {y[2 * p], y[2 * p + 1]};
        C<double> sum = {0.0, 0.0};
        for (int t = 0; t < L.n; ++t) {
            const C<double> M = {L.m_re[t], L.m_im[t]};
            C<double> a = x + yy + M;
            C<double> ia = cinv(a);
            C<double> v = 4.0 * (yy * ia);
            C<double> w = (x * v) * ia;
            C<double> S;
            if (kp.ang_exact) {
                S = exact_S<double>(kp.dim, v, w);
            } else {
                double A = 0.0, Bs = 0.0;
                for (int j = 0; j < kp.npair; ++j) {
                    double r = rcp(q_direct(ang[3 * j], w.r, w.i));
                    A = fma(ang[3 * j + 1], r, A);
                    Bs = fma(ang[3 * j + 2], r, Bs);
                }
                C<double> T2 = {A - w.r * Bs, w.i * Bs};
                C<double> lead = (kp.delta * yy - kp.Omega * (x + M)) * ia - kp.Omega1 * w;
                S = lead + ((v - w) * w) * T2;
            }
            C<double> c = {L.c_re[t], L.c_im[t]};
            sum = sum + (c * ((2.0 * x) * ia)) * (S * cinv(yy + M));
        }
        B[2 * p] = sum.r;
        B[2 * p + 1] = sum.i;
    }
}

// Region 1: eq. 24-25 with the pole at s = -M: k = sqrt(x) cos th +-
// sqrt(-x sin^2 th - M), y = k^2, th in [0, pi], traced on nth samples with
// the two roots matched by continuity; the cut obstructs the real-axis
// contour if a root crosses the positive real y-axis.
__global__ void __launch_bounds__(256)
region_map_kernel(LegTerms L, const double *__restrict__ x, int64_t n, int nth,
                  int *__restrict__ free_out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n;
         p += (int64_t)gridDim.x * blockDim.x) {
        const C<double> xx = {x[2 * p], x[2 * p + 1]};
        const C<double> sx = csqrt_p(xx);
        int obstructed = 0;
        for (int t = 0; t < L.n && !obstructed; ++t) {
            const C<double> M = {L.m_re[t], L.m_im[t]};
            C<double> p1 = {0.0, 0.0}, p2 = {0.0, 0.0};
            for (int i = 0; i < nth && !obstructed; ++i) {
                double th = PI_D() * i / (nth - 1);
                double cs = cos(th), sn = sin(th);
                C<double> r = csqrt_p(C<double>{-xx.r * sn * sn - M.r, -xx.i * sn * sn - M.i});
                C<double> k1 = cs * sx + r, k2 = cs * sx - r;
                C<double> y1 = k1 * k1, y2 = k2 * k2;
                if (i > 0) {
                    if (cabs1(y1 - p1) + cabs1(y2 - p2) > cabs1(y1 - p2) + cabs1(y2 - p1)) {
                        C<double> tmp = y1;
                        y1 = y2;
                        y2 = tmp;
                    }
                    const C<double> prev[2] = {p1, p2}, cur[2] = {y1, y2};
                    for (int b = 0; b < 2; ++b) {
                        double a0 = prev[b].i, a1 = cur[b].i;
                        if ((a0 < 0.0 && a1 >= 0.0) || (a0 > 0.0 && a1 <= 0.0)) {
                            double f = a0 / (a0 - a1);
                            if (prev[b].r + f * (cur[b].r - prev[b].r) > 0.0) obstructed = 1;
                        }
                    }
                }
                p1 = y1;
                p2 = y2;
            }
        }
        free_out[p] = !obstructed;
    }
}

unsigned grid_for(int64_t n)
{
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t b = (n + 255) / 256, cap = (int64_t)sms * 8;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

}  // namespace gfc

using namespace gfc;

extern "C" int gfc_angular_map(const gfc_propagator *prop, const gfc_params *params, double x_re,
                               double x_im, const double *y, int64_t ny, double *B, void *stream)
{
    int rc = check_params_c(params);
    if (rc) return rc;
    if (!prop) return fail(GFC_EINVAL, "propagator is NULL");
    PropConst pc;
    if ((rc = make_prop_c(prop, params, pc))) return rc;
    if (!std::isfinite(x_re) || !std::isfinite(x_im)) return fail(GFC_EINVAL, "x must be finite");
    if (ny < 0) return fail(GFC_EINVAL, "ny < 0");
    if (ny > 0 && (!y || !B)) return fail(GFC_EINVAL, "y and B must be device pointers");
    LegTerms L;
    if ((rc = leg_terms(prop, L))) return rc;
    int dev;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    Tables *T;
    if ((rc = get_tables_c(dev, params->n_radial, params->n_angular, params->dim,
                           params->radial_scale, params->angular_rule, &T, nullptr)))
        return rc;
    KParams kp;
    fill_kparams_c(kp, params, *T, pc);
    DevTables tb = dev_tables_c(*T);
    if (ny == 0) return GFC_OK;
    angular_map_kernel<<<grid_for(ny), 256, 0, (cudaStream_t)stream>>>(kp, tb.ang64, L, x_re,
                                                                        x_im, y, ny, B);
    e = cudaGetLastError();
    return e == cudaSuccess ? GFC_OK : cuda_fail(e, "angular_map launch");
}

extern "C" int gfc_region_map(const gfc_propagator *prop, const double *x, int64_t npts,
                              int32_t *free_out, void *stream)
{
    if (!prop) return fail(GFC_EINVAL, "propagator is NULL");
    gfc_params par;
    gfc_params_default(&par);
    PropConst pc;
    int rc = make_prop_c(prop, &par, pc);
    if (rc) return rc;
    if (npts < 0) return fail(GFC_EINVAL, "npts < 0");
    if (npts > 0 && (!x || !free_out)) return fail(GFC_EINVAL, "x and free_out must be device pointers");
    LegTerms L;
    if ((rc = leg_terms(prop, L))) return rc;
    if (npts == 0) return GFC_OK;
    region_map_kernel<<<grid_for(npts), 256, 0, (cudaStream_t)stream>>>(L, x, npts, 4096,
                                                                         free_out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GFC_OK : cuda_fail(e, "region_map launch");
}
