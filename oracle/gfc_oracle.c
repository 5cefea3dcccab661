/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow, FP64 CPU evaluation of the Taylor-subtracted two-point integral
 *
 *     G(x) = G0(x) - G0(mu2),
 *     G0(x) = K_D * int_C dy (1/2) y^((D-2)/2) int_0^pi dpsi sin^(D-2)(psi)
 *                  P1(y) [P2(x + y - 2 sqrt(x) sqrt(y) cos psi) - P2(y)]
 *
 * on points x = p^2 of the complex plane, written from the paper's recipe:
 *   Step 1 (Sect. 2, eqs. 5-11): hyperspherical reduction to (y, z = cos psi);
 *   Step 2 (eqs. 12-14, 20): BPHZ Taylor subtraction (1 - t^0) at x = 0, in the
 *           combined-fraction form of the third line of eq. 20;
 *   Step 3 (eq. 15, Sect. 5.3 contours C_(2,5), C_3, C_4): deformed radial path;
 *   Step 5 (Sect. 4, "Kernel 2"): non-adaptive Gauss-Legendre quadrature.
 * It is deliberately unoptimised: unpaired angular nodes, nested loops, one
 * complex division per node-eval, Neumaier summation in both loops, threads
 * over points only. Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg load it; the product library never links or calls it.
 *
 * Readings of points where the paper is silent:
 *  - the radial variable is |q| = sqrt(y) on the mapped half-line
 *    |q| = L t/(1-t), t Gauss-Legendre on (0,1) (Lambda^2 -> infinity);
 *  - the default angular rule is Gauss-Legendre in psi on [0,pi] with weight
 *    sin^(D-2) psi (the paper uses tanh-sinh in z with sqrt(1-z^2));
 *  - the radial ray for complex x runs along arg y = arg x (generalising the
 *    paper's regions 2/5 contour 0 -> 15 e^{i arg x});
 *  - a pole of the k-leg that the rotation sweeps is passed by the paper's
 *    detour (straight to the pole, semicircle of radius r, straight out to
 *    R_d e^{i arg x}, R_d = |x| + 20), generalising C_3 / C_4;
 *  - for conjugate-pair legs the k-leg is given the pole in the half-plane of
 *    Im x (the k <-> p-k relabelling is exact for the x = 0 subtraction);
 *  - the subtraction point mu2 enters as the constant shift G0(mu2).
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "gfc_oracle.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef double complex cplx;

/* Planted mistakes, compiled in only by the test that shows the pins can fail
 * (a separate library built with -DORC_MUTANT=n); 0 = the oracle as written.
 *  1 detour half circle on the wrong side     2 no k <-> p-k relabelling
 *  3 q-ray always at arg x / 2                4 K_4 off by a factor 2
 *  5 -x dropped from y - s                     6 weight sin^(D-1) psi
 *  7 dressed mixed term with legs swapped     8 grid without half-cell offset
 *  9 no detour for a ray grazing the k-leg pole
 * 10 a b dropped from the dressed numerator of P(s) - P(y) */
#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

/* ---------------------------------------------------------------------------
 * Gauss-Legendre nodes and weights on [-1, 1] (Abramowitz & Stegun 25.4.29):
 * Newton iteration on P_n from the three-term recurrence, ascending order.
 * ------------------------------------------------------------------------- */
int orc_gauss_legendre(int n, double *x, double *w)
{
    if (n < 1) return ORC_EINVAL;
    for (int i = 0; i < n; ++i) {
        /* i-th root counted from +1 downwards */
        double r = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = r;
            for (int k = 2; k <= n; ++k) {
                double pk = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (n == 1) { p1 = r; p0 = 1.0; }
            dp = n * (r * p1 - p0) / (r * r - 1.0);
            double dr = p1 / dp;
            r -= dr;
            if (fabs(dr) < 1e-16) break;
        }
        /* recompute the derivative at the converged root */
        double p0 = 1.0, p1 = r;
        for (int k = 2; k <= n; ++k) {
            double pk = ((2.0 * k - 1.0) * r * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = pk;
        }
        if (n == 1) { p1 = r; p0 = 1.0; }
        dp = n * (r * p1 - p0) / (r * r - 1.0);
        x[n - 1 - i] = r;
        w[n - 1 - i] = 2.0 / ((1.0 - r * r) * dp * dp);
    }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Neumaier (improved Kahan) complex summation.
 * ------------------------------------------------------------------------- */
typedef struct { double s_re, c_re, s_im, c_im; } nsum;

static void nsum_add1(double *s, double *c, double v)
{
    double t = *s + v;
    if (fabs(*s) >= fabs(v)) *c += (*s - t) + v;
    else                     *c += (v - t) + *s;
    *s = t;
}

static void nsum_add(nsum *a, cplx v)
{
    nsum_add1(&a->s_re, &a->c_re, creal(v));
    nsum_add1(&a->s_im, &a->c_im, cimag(v));
}

static cplx nsum_get(const nsum *a) { return (a->s_re + a->c_re) + I * (a->s_im + a->c_im); }

/* ---------------------------------------------------------------------------
 * Propagators on one leg.  PL_POLE: 1/(s + M2) with complex M2.
 * PL_DRESSED: (s + a)/(s^2 + b s + c).
 * ------------------------------------------------------------------------- */
enum { PL_POLE = 0, PL_DRESSED = 1 };
typedef struct { int form; cplx M2; double a, b, c; } leg;

static cplx leg_eval(const leg *L, cplx s)
{
    if (L->form == PL_POLE) return 1.0 / (s + L->M2);
    return (s + L->a) / (s * s + L->b * s + L->c);
}

/* P(s) - P(y) with (y - s) factored out as in the third line of eq. 20, so the
 * Taylor subtraction is carried out algebraically, not by cancellation. */
static cplx leg_diff(const leg *L, cplx s, cplx y, cplx y_minus_s)
{
    if (L->form == PL_POLE) return y_minus_s / ((s + L->M2) * (y + L->M2));
    cplx num = s * y + L->a * (s + y) + (ORC_MUTANT == 10 ? 0.0 : L->a * L->b) - L->c;
    return y_minus_s * num / ((s * s + L->b * s + L->c) * (y * y + L->b * y + L->c));
}

/* ---------------------------------------------------------------------------
 * Contours: a list of nodes (y_k, dy_k, sq_k) with sq_k the branch of sqrt(y_k)
 * that the deformation carries along (it enters the D = 3 measure, which is
 * odd under q -> -q).  The measure (1/2) y^((D-2)/2) dy equals q^(D-1) dq.
 * ------------------------------------------------------------------------- */
typedef struct { cplx *y, *dy, *sq; int n, cap; } nodes;

static void nodes_push(nodes *N, cplx y, cplx dy, cplx sq)
{
    N->y[N->n] = y;
    N->dy[N->n] = dy;
    N->sq[N->n] = sq;
    N->n++;
}

typedef struct {
    int dim, n_r, n_a;
    double L, r_detour;
    double *gr_x, *gr_w;     /* GL on [-1,1], n_r nodes (radial) */
    double *gs_x, *gs_w;     /* GL on [-1,1], n_r/4 nodes (detour segments) */
    double *gt_x, *gt_w;     /* GL on [-1,1], n_r/2 nodes (clustered rule's tail) */
    int radial_rule;
    cplx ppoles[4];          /* poles of the propagator as given (y-plane) */
    int nppoles;
    double *psi, *wpsi;      /* angular: psi_j, w_j sin^(D-2) psi_j */
    double *cpsi;            /* cos psi_j */
    int exact;               /* psi integral in closed form */
    double K_D;
} rules;

/* The clustered radial rule (near-axis accuracy): the propagator's poles y_p
 * give q-plane points +-sqrt(y_p); the one closest in angle to the ray
 * arg q = theta, with d < 0.75 c (within ~37 degrees; a reading: the paper
 * gives no rule), has projection c and distance d from the ray. The ray then takes n_r/4 GL nodes on each of [0, c] and [c, 2c],
 * mapped by |q| = c + d sinh(s) (s from -asinh(c/d) to 0, and from 0 to
 * asinh(c/d)), which packs nodes within ~d of the near-singular point, and
 * n_r/2 GL nodes on the mapped half-line |q| = 2c + L t/(1-t). Returns 0 when
 * no pole qualifies (the plain mapped ray is used). */
static int cluster_point(const rules *R, double theta, double *c, double *d)
{
    cplx e = cexp(-I * theta);
    double best = 1.0;
    int found = 0;
    for (int i = 0; i < R->nppoles; ++i) {
        for (int sg = -1; sg <= 1; sg += 2) {
            cplx z = sg * csqrt(R->ppoles[i]) * e;
            double rs = creal(z), ds = fabs(cimag(z));
            if (rs > 0.0 && ds < 0.75 * rs && ds / rs < best) {
                best = ds / rs;
                *c = rs;
                *d = ds;
                found = 1;
            }
        }
    }
    if (found && *d < 1e-12 * *c) *d = 1e-12 * *c;
    return found;
}

static void add_ray_clustered(nodes *N, const rules *R, double theta, double c, double d)
{
    cplx e = cexp(I * theta);
    int ns = R->n_r / 4, nt = R->n_r / 2;
    double eta = asinh(c / d);
    for (int panel = 0; panel < 2; ++panel) {
        for (int k = 0; k < ns; ++k) {
            double t = 0.5 * (R->gs_x[k] + 1.0), wt = 0.5 * R->gs_w[k];
            double sv = panel == 0 ? eta * (t - 1.0) : eta * t;
            double rho = c + d * sinh(sv), drho = d * cosh(sv) * eta * wt;
            cplx q = rho * e;
            nodes_push(N, q * q, 2.0 * q * e * drho, q);
        }
    }
    for (int k = 0; k < nt; ++k) {
        double t = 0.5 * (R->gt_x[k] + 1.0), wt = 0.5 * R->gt_w[k];
        double rho = 2.0 * c + R->L * t / (1.0 - t);
        double drho = R->L / ((1.0 - t) * (1.0 - t)) * wt;
        cplx q = rho * e;
        nodes_push(N, q * q, 2.0 * q * e * drho, q);
    }
}

/* q-ray from |q| = rho0 to infinity along arg q = theta (so arg y = 2 theta):
 * |q| = rho0 + L t/(1-t), t = GL on (0,1); y = q^2, dy = 2 q dq. */
static void add_ray(nodes *N, const rules *R, double theta, double rho0)
{
    cplx e = cexp(I * theta);
    for (int k = 0; k < R->n_r; ++k) {
        double t = 0.5 * (R->gr_x[k] + 1.0), wt = 0.5 * R->gr_w[k];
        double rho = rho0 + R->L * t / (1.0 - t);
        double drho = R->L / ((1.0 - t) * (1.0 - t)) * wt;
        cplx q = rho * e;
        nodes_push(N, q * q, 2.0 * q * e * drho, q);
    }
}

/* straight segment in the q-plane from 0 to q1 (a radial segment of the
 * y-plane from 0 to q1^2), n_r/4 GL nodes; smooth at y = 0 in every D */
static void add_qsegment(nodes *N, const rules *R, cplx q1)
{
    int ns = R->n_r / 4;
    for (int k = 0; k < ns; ++k) {
        double t = 0.5 * (R->gs_x[k] + 1.0), wt = 0.5 * R->gs_w[k];
        cplx q = q1 * t;
        nodes_push(N, q * q, 2.0 * q * q1 * wt, q);
    }
}

/* straight segment y0 -> y1 in the y-plane, n_r/4 GL nodes, principal sqrt */
static void add_segment(nodes *N, const rules *R, cplx y0, cplx y1)
{
    int ns = R->n_r / 4;
    for (int k = 0; k < ns; ++k) {
        double t = 0.5 * (R->gs_x[k] + 1.0), wt = 0.5 * R->gs_w[k];
        cplx y = y0 + (y1 - y0) * t;
        nodes_push(N, y, (y1 - y0) * wt, csqrt(y));
    }
}

/* arc y = c + r e^{i theta}, theta from th0 to th1, n_r/4 GL nodes */
static void add_arc(nodes *N, const rules *R, cplx c, double r, double th0, double th1)
{
    int ns = R->n_r / 4;
    for (int k = 0; k < ns; ++k) {
        double t = 0.5 * (R->gs_x[k] + 1.0), wt = 0.5 * R->gs_w[k];
        double th = th0 + (th1 - th0) * t;
        cplx e = cexp(I * th);
        cplx y = c + r * e;
        nodes_push(N, y, I * r * e * (th1 - th0) * wt, csqrt(y));
    }
}

/* The paper's detour (contours C_3, C_4 of Sect. 5.3, generalised): straight
 * along the direction of the pole yp to |yp| - r, a half circle around yp that
 * leaves yp on the side of the path where the real y-axis had it, straight to
 * R_d e^{i phi}, then the ray to infinity. */
static void add_detour(nodes *N, const rules *R, cplx x, cplx yp)
{
    double phi = carg(x);
    double ap = cabs(yp), r = R->r_detour;
    cplx u = yp / ap;
    double sg = cimag(yp) > 0 ? 1.0 : -1.0;
    if (ORC_MUTANT == 1) sg = -sg;
    double th0 = carg(-u);
    double Rd = cabs(x) + 20.0;
    add_qsegment(N, R, csqrt((ap - r) * u));
    add_arc(N, R, yp, r, th0, th0 + sg * M_PI);
    add_segment(N, R, (ap + r) * u, Rd * cexp(I * phi));
    add_ray(N, R, 0.5 * phi, sqrt(Rd));
}

/* Does rotating the positive real q-axis to arg q = theta sweep the point qp? */
static int q_swept(cplx qp, double theta)
{
    double a = carg(qp);
    return (0.0 < a && a < theta) || (theta < a && a < 0.0);
}

/* The two q-rays on which y = q^2 runs along arg y = arg x (Step 3 read in the
 * q-plane): theta = phi/2, or the opposite direction phi/2 - pi sgn(phi).
 * Returns the first that sweeps none of the poles +-sqrt(y_p) of either leg,
 * or NAN when both do (then the detour is needed). */
static double choose_ray(double phi, const cplx *ypoles, int npoles)
{
    double cand[2] = {0.5 * phi, 0.5 * phi - (phi >= 0.0 ? M_PI : -M_PI)};
    if (ORC_MUTANT == 3) return cand[0];
    for (int c = 0; c < 2; ++c) {
        int bad = 0;
        for (int i = 0; i < npoles && !bad; ++i) {
            cplx qp = csqrt(ypoles[i]);
            bad = q_swept(qp, cand[c]) || q_swept(-qp, cand[c]);
        }
        if (!bad) return cand[c];
    }
    return NAN;
}

/* ---------------------------------------------------------------------------
 * The psi integral in closed form. With s = x + y - B cos psi, B = 2 sqrt(x)
 * sqrt(y), a pole leg 1/(s + M2) has A = x + y + M2 and
 *   int_0^pi sin^2 psi dpsi/(A - B cos psi) = pi/(A (1 + sqrt(1 - B^2/A^2)))
 *   int_0^pi sin psi dpsi/(A - B cos psi) = (2/A) artanh(B/A)/(B/A)
 * (the first by the substitution t = tan(psi/2) and residues, the second by
 * z = cos psi), principal branches, which continue the real-positive case
 * analytically off B^2/A^2 in [1, inf). A dressed leg is split into its two
 * poles: (s + a)/((s - r1)(s - r2)) = R1/(s - r1) + R2/(s - r2).
 * ------------------------------------------------------------------------- */
static cplx pole_angular(int dim, cplx A, cplx B2)
{
    cplx w = B2 / (A * A);
    if (dim == 4) return M_PI / (A * (1.0 + csqrt(1.0 - w)));
    cplx z = csqrt(w);
    return cabs(z) < 1e-8 ? 2.0 / A * (1.0 + w / 3.0) : 2.0 / A * catanh(z) / z;
}

/* int_0^pi sin^(D-2) psi [P2(s(psi)) - P2(y)] dpsi for one leg */
static cplx leg_angular(const leg *L, int dim, cplx x, cplx y)
{
    cplx B2 = 4.0 * x * y;
    double wtot = dim == 4 ? 0.5 * M_PI : 2.0;
    if (L->form == PL_POLE) return pole_angular(dim, x + y + L->M2, B2) - wtot * leg_eval(L, y);
    double disc = 4.0 * L->c - L->b * L->b;
    cplx r1 = 0.5 * (-L->b + I * sqrt(disc)), r2 = conj(r1);
    cplx R1 = (r1 + L->a) / (r1 - r2), R2 = (r2 + L->a) / (r2 - r1);
    return R1 * pole_angular(dim, x + y - r1, B2) + R2 * pole_angular(dim, x + y - r2, B2)
           - wtot * leg_eval(L, y);
}

/* ---------------------------------------------------------------------------
 * One term: coef * int_C dy 1/2 y^((D-2)/2) int dpsi w(psi) P1(y)[P2(s) - P2(y)]
 * ------------------------------------------------------------------------- */
static void term_sum(const rules *R, cplx x, cplx coef, const leg *P1, const leg *P2,
                     const nodes *N, nsum *outer, double *abs_sum)
{
    cplx sx = csqrt(x);
    for (int k = 0; k < N->n; ++k) {
        cplx y = N->y[k];
        cplx sy = N->sq[k];
        cplx meas = 0.5 * (R->dim == 4 ? y : sy) * N->dy[k];
        cplx p1 = leg_eval(P1, y);
        nsum inner = {0, 0, 0, 0};
        double ainner = 0.0;
        if (R->exact) {
            cplx f = p1 * leg_angular(P2, R->dim, x, y);
            nsum_add(&inner, f);
            ainner = cabs(f);
        }
        for (int j = 0; j < (R->exact ? 0 : R->n_a); ++j) {
            cplx ymS = (ORC_MUTANT == 5 ? 0.0 : -x) + 2.0 * sx * sy * R->cpsi[j];  /* y - s */
            cplx s = y - ymS;
            cplx f = R->wpsi[j] * p1 * leg_diff(P2, s, y, ymS);
            nsum_add(&inner, f);
            ainner += cabs(f);
        }
        cplx v = coef * meas * nsum_get(&inner);
        nsum_add(outer, v);
        *abs_sum += cabs(coef * meas) * ainner;
    }
}

/* poles y_p of one leg in the y-plane */
static int leg_poles(const leg *L, cplx *out)
{
    if (L->form == PL_POLE) { out[0] = -L->M2; return 1; }
    double disc = 4.0 * L->c - L->b * L->b;
    out[0] = 0.5 * (-L->b + I * sqrt(disc));
    out[1] = conj(out[0]);
    return 2;
}

/* Distance from the y-ray along arg y = phi to the point yp. */
static double ray_distance(cplx yp, double phi)
{
    double d = fabs(carg(yp) - phi);
    if (d > M_PI) d = 2.0 * M_PI - d;
    return d < 0.5 * M_PI ? cabs(yp) * sin(d) : cabs(yp);
}

/* Contour of one term: a q-ray sweeping no pole of either leg if there is one,
 * otherwise the detour around the pole of the k-leg (which the caller has put
 * in the half-plane of Im x). For legs with different poles the detour is also
 * taken when the ray would pass within 2 r of the k-leg pole. */
static void term_contour(nodes *N, const rules *R, cplx x, const leg *P1, const leg *P2)
{
    cplx poles[4];
    int np = leg_poles(P1, poles);
    np += leg_poles(P2, poles + np);
    double phi = carg(x);
    double theta = choose_ray(phi, poles, np);
    int pair = P1->form == PL_POLE && P2->form == PL_POLE && P1->M2 != P2->M2;
    if (pair && !isnan(theta) && ORC_MUTANT != 9 &&
        ray_distance(-P1->M2, phi) < 2.0 * R->r_detour && cimag(-P1->M2) * cimag(x) > 0.0)
        theta = NAN;
    N->n = 0;
    double c, d;
    if (!isnan(theta) && R->radial_rule == ORC_RAD_CLUSTERED && cluster_point(R, theta, &c, &d))
        add_ray_clustered(N, R, theta, c, d);
    else if (!isnan(theta))
        add_ray(N, R, theta, 0.0);
    else
        add_detour(N, R, x, -P1->M2);
}

static int G0_point(const orc_prop *P, const rules *R, cplx x, cplx *G0, double *kappa,
                    nodes *N)
{
    double phi = carg(x);
    nsum acc = {0, 0, 0, 0};
    double asum = 0.0;

    if (P->kind == ORC_PROP_SCALAR) {
        leg l = {PL_POLE, P->m2, 0, 0, 0};
        term_contour(N, R, x, &l, &l);
        term_sum(R, x, 1.0, &l, &l, N, &acc, &asum);
    } else if (P->kind == ORC_PROP_CPAIR) {
        cplx Ma = P->mk2_re + I * P->mk2_im, Mb = P->mq2_re + I * P->mq2_im;
        /* k-leg carries the pole -M^2 lying in the half-plane of Im x */
        cplx Mk = Ma, Mq = Mb;
        if (cimag(x) > 0.0 && cimag(-Ma) < 0.0 && ORC_MUTANT != 2) { Mk = Mb; Mq = Ma; }
        if (cimag(x) < 0.0 && cimag(-Ma) > 0.0 && ORC_MUTANT != 2) { Mk = Mb; Mq = Ma; }
        leg lk = {PL_POLE, Mk, 0, 0, 0}, lq = {PL_POLE, Mq, 0, 0, 0};
        term_contour(N, R, x, &lk, &lq);
        term_sum(R, x, 1.0, &lk, &lq, N, &acc, &asum);
    } else if (P->kind == ORC_PROP_DRESSED) {
        double a = P->a, b = P->b, c = P->c;
        double disc = 4.0 * c - b * b;
        if (!(disc > 0.0)) return ORC_EINVAL;
        cplx yp = 0.5 * (-b + I * sqrt(disc)), ym = conj(yp);
        if (fabs(phi) < carg(yp)) {
            /* nothing swept: the full dressed integrand on the ray */
            leg ld = {PL_DRESSED, 0, a, b, c};
            term_contour(N, R, x, &ld, &ld);
            term_sum(R, x, 1.0, &ld, &ld, N, &acc, &asum);
        } else {
            /* partial fractions D(s) = R+/(s-y+) + R-/(s-y-) */
            cplx Rp = (yp + a) / (yp - ym), Rm = (ym + a) / (ym - yp);
            leg lp = {PL_POLE, -yp, 0, 0, 0}, lm = {PL_POLE, -ym, 0, 0, 0};
            term_contour(N, R, x, &lp, &lp);
            term_sum(R, x, Rp * Rp, &lp, &lp, N, &acc, &asum);
            term_contour(N, R, x, &lm, &lm);
            term_sum(R, x, Rm * Rm, &lm, &lm, N, &acc, &asum);
            /* mixed term 2 R+ R- T(k: pole in the half-plane of Im x) */
            const leg *lk = (cimag(x) > 0.0) != (ORC_MUTANT == 7) ? &lp : &lm;
            const leg *lq = lk == &lp ? &lm : &lp;
            term_contour(N, R, x, lk, lq);
            term_sum(R, x, 2.0 * Rp * Rm, lk, lq, N, &acc, &asum);
        }
    } else {
        return ORC_EINVAL;
    }
    cplx s = nsum_get(&acc);
    *G0 = R->K_D * s;
    if (kappa) *kappa = cabs(s) > 0.0 ? asum / cabs(s) : INFINITY;
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Angular rules (Sect. 4: the angular integral by tanh-sinh quadrature in
 * z = cos psi, Gauss-Chebyshev rules of both kinds as a check). All four
 * integrate int_0^pi f(cos psi) sin^(D-2) psi dpsi, i.e. int_-1^1 f(z)
 * (1 - z^2)^((D-3)/2) dz, and return z_j = cos psi_j with weights w_j.
 *  - GL: Gauss-Legendre in psi on [0, pi], w = (pi/2) w_GL sin^(D-2) psi.
 *  - tanh-sinh: z = tanh(pi/2 sinh s), s = k h, k = -N..N (n = 2N + 1),
 *    dz = (pi/2) cosh s / cosh^2(pi/2 sinh s) ds, trapezoid in s; the step
 *    h = 3/N spans s in [-3, 3] (the paper gives the order only), where
 *    1 - |z| ~ 1e-14. (1 - z^2)^(1/2) = 1/cosh(pi/2 sinh s) exactly.
 *  - Chebyshev 1st kind: int g(z)/sqrt(1-z^2) dz ~ (pi/n) sum g(cos psi_j),
 *    psi_j = (j - 1/2) pi/n, so w_j = (pi/n) sin^(D-2) psi_j.
 *  - Chebyshev 2nd kind: int g(z) sqrt(1-z^2) dz ~ pi/(n+1) sum sin^2 psi_j
 *    g(cos psi_j), psi_j = j pi/(n+1), so w_j = pi/(n+1) sin^(D-2) psi_j.
 * ------------------------------------------------------------------------- */
int orc_angular_rule(int rule, int n, int dim, double *z, double *w)
{
    if (n < 2 || (dim != 3 && dim != 4)) return ORC_EINVAL;
    if (rule == ORC_ANG_GL) {
        double *gx = malloc(sizeof(double) * n), *gw = malloc(sizeof(double) * n);
        if (!gx || !gw) { free(gx); free(gw); return ORC_ENOMEM; }
        orc_gauss_legendre(n, gx, gw);
        for (int j = 0; j < n; ++j) {
            double psi = 0.5 * M_PI * (gx[j] + 1.0), sn = sin(psi);
            z[j] = cos(psi);
            w[j] = 0.5 * M_PI * gw[j] * (dim == 4 ? sn * sn : sn);
            if (ORC_MUTANT == 6) w[j] *= sn;
        }
        free(gx);
        free(gw);
        return ORC_OK;
    }
    if (rule == ORC_ANG_TANH_SINH) {
        if (n % 2 == 0 || n < 3) return ORC_EINVAL;
        int N = (n - 1) / 2;
        double h = 3.0 / N;
        for (int k = -N; k <= N; ++k) {
            double s = k * h, u = 0.5 * M_PI * sinh(s), cu = cosh(u);
            double dz = h * 0.5 * M_PI * cosh(s) / (cu * cu);
            z[k + N] = tanh(u);
            w[k + N] = dim == 4 ? dz / cu : dz;
        }
        return ORC_OK;
    }
    if (rule == ORC_ANG_CHEB1 || rule == ORC_ANG_CHEB2) {
        for (int j = 1; j <= n; ++j) {
            double psi = rule == ORC_ANG_CHEB1 ? (j - 0.5) * M_PI / n : j * M_PI / (n + 1);
            double sn = sin(psi), c = rule == ORC_ANG_CHEB1 ? M_PI / n : M_PI / (n + 1);
            z[j - 1] = cos(psi);
            w[j - 1] = c * (dim == 4 ? sn * sn : sn);
        }
        return ORC_OK;
    }
    return ORC_EINVAL;
}

/* ---------------------------------------------------------------------------
 * Rules setup / teardown.
 * ------------------------------------------------------------------------- */
static void rules_free(rules *R)
{
    free(R->gr_x); free(R->gr_w); free(R->gs_x); free(R->gs_w); free(R->gt_x); free(R->gt_w);
    free(R->psi); free(R->wpsi); free(R->cpsi);
}

static int rules_init(rules *R, const orc_params *Q)
{
    memset(R, 0, sizeof *R);
    if (Q->dim != 3 && Q->dim != 4) return ORC_EINVAL;
    if (Q->n_angular < 2) return ORC_EINVAL;
    if (Q->angular_rule == ORC_ANG_TANH_SINH && Q->n_angular % 2 == 0) return ORC_EINVAL;
    if (Q->angular_rule < ORC_ANG_GL || Q->angular_rule > ORC_ANG_EXACT) return ORC_EINVAL;
    if (Q->radial_rule != ORC_RAD_MAPPED && Q->radial_rule != ORC_RAD_CLUSTERED) return ORC_EINVAL;
    if (Q->n_radial < 4 || Q->n_radial % 4) return ORC_EINVAL;
    if (!(Q->radial_scale > 0.0) || !(Q->detour_radius > 0.0)) return ORC_EINVAL;
    R->dim = Q->dim;
    R->n_r = Q->n_radial;
    R->n_a = Q->n_angular;
    R->L = Q->radial_scale;
    R->r_detour = Q->detour_radius;
    int ns = R->n_r / 4;
    R->gr_x = malloc(sizeof(double) * R->n_r);
    R->gr_w = malloc(sizeof(double) * R->n_r);
    R->gs_x = malloc(sizeof(double) * ns);
    R->gs_w = malloc(sizeof(double) * ns);
    R->psi = malloc(sizeof(double) * R->n_a);
    R->wpsi = malloc(sizeof(double) * R->n_a);
    R->cpsi = malloc(sizeof(double) * R->n_a);
    R->gt_x = malloc(sizeof(double) * (R->n_r / 2));
    R->gt_w = malloc(sizeof(double) * (R->n_r / 2));
    orc_gauss_legendre(R->n_r, R->gr_x, R->gr_w);
    orc_gauss_legendre(ns, R->gs_x, R->gs_w);
    orc_gauss_legendre(R->n_r / 2, R->gt_x, R->gt_w);
    R->radial_rule = Q->radial_rule;
    R->exact = Q->angular_rule == ORC_ANG_EXACT;
    int rc = orc_angular_rule(R->exact ? ORC_ANG_GL : Q->angular_rule, R->n_a, R->dim, R->cpsi,
                              R->wpsi);
    if (rc != ORC_OK) {
        rules_free(R);
        return rc;
    }
    for (int j = 0; j < R->n_a; ++j) R->psi[j] = acos(R->cpsi[j]);
    /* K_D = S_(D-2) / (2 pi)^D: K_4 = 4 pi/(2 pi)^4, K_3 = 2 pi/(2 pi)^3 (eq. 11) */
    R->K_D = R->dim == 4 ? 4.0 * M_PI / pow(2.0 * M_PI, 4) : 2.0 * M_PI / pow(2.0 * M_PI, 3);
    if (ORC_MUTANT == 4 && R->dim == 4) R->K_D *= 2.0;
    return ORC_OK;
}


static int nodes_alloc(nodes *N, int n_r)
{
    N->cap = 2 * n_r + 8;   /* detour: 3 * n_r/4 + n_r */
    N->n = 0;
    N->y = malloc(sizeof(cplx) * N->cap);
    N->dy = malloc(sizeof(cplx) * N->cap);
    N->sq = malloc(sizeof(cplx) * N->cap);
    return (N->y && N->dy && N->sq) ? ORC_OK : ORC_ENOMEM;
}

static void nodes_free(nodes *N) { free(N->y); free(N->dy); free(N->sq); }

/* ---------------------------------------------------------------------------
 * Threaded driver over points.
 * ------------------------------------------------------------------------- */
typedef struct {
    const orc_prop *P;
    const rules *R;
    const double *x;
    double *G, *kappa;
    long n, start, stride;
    cplx G0mu;
    int status;
} job;

static void *worker(void *arg)
{
    job *J = arg;
    nodes N;
    if (nodes_alloc(&N, J->R->n_r) != ORC_OK) { J->status = ORC_ENOMEM; return NULL; }
    for (long i = J->start; i < J->n; i += J->stride) {
        cplx x = J->x[2 * i] + I * J->x[2 * i + 1];
        cplx g0;
        double kap = 0.0;
        int st = G0_point(J->P, J->R, x, &g0, &kap, &N);
        if (st != ORC_OK) { J->status = st; break; }
        cplx g = g0 - J->G0mu;
        J->G[2 * i] = creal(g);
        J->G[2 * i + 1] = cimag(g);
        if (J->kappa) J->kappa[i] = kap;
    }
    nodes_free(&N);
    return NULL;
}

static int check_prop(const orc_prop *P)
{
    if (P->kind == ORC_PROP_SCALAR) return P->m2 > 0.0 ? ORC_OK : ORC_EINVAL;
    if (P->kind == ORC_PROP_CPAIR) {
        /* conjugate pair with poles off the real axis */
        if (P->mk2_re != P->mq2_re || P->mk2_im != -P->mq2_im || P->mk2_im == 0.0) return ORC_EINVAL;
        return ORC_OK;
    }
    if (P->kind == ORC_PROP_DRESSED) return (4.0 * P->c - P->b * P->b > 0.0) ? ORC_OK : ORC_EINVAL;
    return ORC_EINVAL;
}

int orc_eval_points(const orc_prop *P, const orc_params *Q, const double *x, long npts,
                    double *G, double *kappa, int nthreads)
{
    if (!P || !Q || (npts > 0 && (!x || !G))) return ORC_EINVAL;
    if (check_prop(P) != ORC_OK) return ORC_EINVAL;
    for (long i = 0; i < npts; ++i) {
        /* the method is undefined on the negative real axis (the cut side) */
        if (x[2 * i + 1] == 0.0 && x[2 * i] < 0.0) return ORC_EINVAL;
        if (!isfinite(x[2 * i]) || !isfinite(x[2 * i + 1])) return ORC_EINVAL;
    }
    if (Q->mu2 < 0.0) return ORC_EINVAL;
    rules R;
    int st = rules_init(&R, Q);
    if (st != ORC_OK) return st;
    /* the half circle must stay well clear of the origin */
    double pole_abs = P->kind == ORC_PROP_CPAIR ? sqrt(P->mk2_re * P->mk2_re + P->mk2_im * P->mk2_im)
                    : P->kind == ORC_PROP_DRESSED ? sqrt(P->c) : INFINITY;
    if (!(R.r_detour < 0.5 * pole_abs)) {
        rules_free(&R);
        return ORC_EINVAL;
    }
    /* the propagator's poles, for the clustered radial rule */
    if (P->kind == ORC_PROP_SCALAR) {
        R.ppoles[0] = -P->m2;
        R.nppoles = 1;
    } else if (P->kind == ORC_PROP_CPAIR) {
        R.ppoles[0] = -(P->mk2_re + I * P->mk2_im);
        R.ppoles[1] = -(P->mq2_re + I * P->mq2_im);
        R.nppoles = 2;
    } else if (4.0 * P->c - P->b * P->b > 0.0) {
        R.ppoles[0] = 0.5 * (-P->b + I * sqrt(4.0 * P->c - P->b * P->b));
        R.ppoles[1] = conj(R.ppoles[0]);
        R.nppoles = 2;
    }

    /* G0(mu2) on the real axis with the same rules */
    cplx g0mu = 0.0;
    {
        nodes N;
        if (nodes_alloc(&N, R.n_r) != ORC_OK) { rules_free(&R); return ORC_ENOMEM; }
        st = G0_point(P, &R, Q->mu2 + 0.0 * I, &g0mu, NULL, &N);
        nodes_free(&N);
        if (st != ORC_OK) { rules_free(&R); return st; }
    }

    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (npts < nthreads) nthreads = npts > 0 ? (int)npts : 1;
    pthread_t th[256];
    job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = (job){P, &R, x, G, kappa, npts, t, nthreads, g0mu, ORC_OK};
        pthread_create(&th[t], NULL, worker, &jobs[t]);
    }
    st = ORC_OK;
    for (int t = 0; t < nthreads; ++t) {
        pthread_join(th[t], NULL);
        if (jobs[t].status != ORC_OK) st = jobs[t].status;
    }
    rules_free(&R);
    return st;
}

/* Step 4 / Kernel 1 (Sect. 4): a homogeneous M x N grid over the rectangle,
 * cell-centred (half-cell offset), real index i < m, imaginary index j < n,
 * stored at [i*n + j]. */
int orc_grid_points(double re0, double re1, double im0, double im1, int m, int n, double *x)
{
    if (m < 1 || n < 1 || !x) return ORC_EINVAL;
    double dre = (re1 - re0) / m, dim = (im1 - im0) / n;
    double half = ORC_MUTANT == 8 ? 0.0 : 0.5;
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            x[2 * ((long)i * n + j)] = re0 + (i + half) * dre;
            x[2 * ((long)i * n + j) + 1] = im0 + (j + half) * dim;
        }
    return ORC_OK;
}

/* ---------------------------------------------------------------------------
 * Step 3 diagnostics (Sect. 5, Figs. 1-2).
 * ------------------------------------------------------------------------- */
/* the (p-k) leg as given by the caller (no relabelling) */
static int given_q_leg(const orc_prop *P, leg *L)
{
    if (P->kind == ORC_PROP_SCALAR) { leg l = {PL_POLE, P->m2, 0, 0, 0}; *L = l; return ORC_OK; }
    if (P->kind == ORC_PROP_CPAIR) {
        leg l = {PL_POLE, P->mq2_re + I * P->mq2_im, 0, 0, 0};
        *L = l;
        return ORC_OK;
    }
    if (P->kind == ORC_PROP_DRESSED && 4.0 * P->c - P->b * P->b > 0.0) {
        leg l = {PL_DRESSED, 0, P->a, P->b, P->c};
        *L = l;
        return ORC_OK;
    }
    return ORC_EINVAL;
}

int orc_angular_map(const orc_prop *P, const orc_params *Q, double xr, double xi,
                    const double *y, long ny, double *B)
{
    leg L;
    if (given_q_leg(P, &L) != ORC_OK || ny < 0) return ORC_EINVAL;
    rules R;
    int rc = rules_init(&R, Q);
    if (rc != ORC_OK) return rc;
    cplx x = xr + I * xi;
    for (long i = 0; i < ny; ++i) {
        cplx yy = y[2 * i] + I * y[2 * i + 1];
        cplx b;
        if (R.exact) {
            b = leg_angular(&L, R.dim, x, yy);
        } else {
            /* the plain sum over the rule's nodes; only x y enters s */
            cplx sxy = csqrt(x * yy), py = leg_eval(&L, yy);
            nsum acc = {0, 0, 0, 0};
            for (int j = 0; j < R.n_a; ++j) {
                cplx s = x + yy - 2.0 * sxy * R.cpsi[j];
                nsum_add(&acc, R.wpsi[j] * (leg_eval(&L, s) - py));
            }
            b = nsum_get(&acc);
        }
        B[2 * i] = creal(b);
        B[2 * i + 1] = cimag(b);
    }
    rules_free(&R);
    return ORC_OK;
}

/* Does some y > 0 give w = 4 x y/(x + y + M2)^2 real and >= 1 (then
 * cos^2 psi = 1/w puts a pole of 1/(s + M2) on the angular range)? The scan
 * y = u/(1 - u), u on a uniform grid of (0, 1), looks for sign changes of
 * Im w and interpolates Re w there. */
static int pole_obstructs(cplx x, cplx M2)
{
    const int K = 16384;
    /* x and M2 real: w is real for every real y and the pole condition
     * cos psi = a/b (b = 2 sqrt(x y)) holds only where a = x + y + M2 = 0,
     * i.e. at y = -x - M2 when that is positive (the cut side of the axis) */
    if (cimag(x) == 0.0 && cimag(M2) == 0.0) return creal(x) < 0.0 && -creal(x) - creal(M2) > 0.0;
    double pim = 0.0, pre = 0.0;
    for (int k = 0; k < K; ++k) {
        double u = (k + 0.5) / K, yv = u / (1.0 - u);
        cplx a = x + yv + M2, w = 4.0 * x * yv / (a * a);
        double wi = cimag(w), wr = creal(w);
        if (k > 0 && ((pim < 0.0 && wi >= 0.0) || (pim > 0.0 && wi <= 0.0))) {
            double f = pim / (pim - wi);
            if (pre + f * (wr - pre) >= 1.0) return 1;
        }
        pim = wi;
        pre = wr;
    }
    return 0;
}

int orc_region_map(const orc_prop *P, const double *x, long n, int *free_out)
{
    leg L;
    if (given_q_leg(P, &L) != ORC_OK || n < 0) return ORC_EINVAL;
    cplx M[2];
    int nm = 1;
    if (L.form == PL_POLE) {
        M[0] = L.M2;
    } else {
        double disc = 4.0 * L.c - L.b * L.b;
        cplx r1 = 0.5 * (-L.b + I * sqrt(disc));
        M[0] = -r1;
        M[1] = -conj(r1);
        nm = 2;
    }
    for (long i = 0; i < n; ++i) {
        cplx xx = x[2 * i] + I * x[2 * i + 1];
        int obstructed = 0;
        for (int t = 0; t < nm && !obstructed; ++t) obstructed = pole_obstructs(xx, M[t]);
        free_out[i] = !obstructed;
    }
    return ORC_OK;
}
