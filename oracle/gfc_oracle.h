/*
 * ORACLE — test infrastructure only (see gfc_oracle.c). Its own definitions;
 * it shares no header, type or helper with the product library.
 */
#ifndef GFC_ORACLE_H
#define GFC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };
enum { ORC_PROP_SCALAR = 0, ORC_PROP_CPAIR = 1, ORC_PROP_DRESSED = 2 };
/* angular rules (Sect. 4): Gauss-Legendre in psi (default), tanh-sinh in
 * z = cos psi (the paper's), Gauss-Chebyshev of the first and second kind */
enum { ORC_ANG_GL = 0, ORC_ANG_TANH_SINH = 1, ORC_ANG_CHEB1 = 2, ORC_ANG_CHEB2 = 3,
       ORC_ANG_EXACT = 4 /* the psi integral in closed form (no angular nodes) */ };
/* radial rules of the rays from q = 0: the mapped half-line, or three panels
 * sinh-clustered at the propagator pole nearest the ray */
enum { ORC_RAD_MAPPED = 0, ORC_RAD_CLUSTERED = 1 };

typedef struct {
    int kind;
    double m2;                  /* SCALAR: 1/(s + m2) on both legs            */
    double mk2_re, mk2_im;      /* CPAIR: k-leg 1/(s + Mk2) as printed        */
    double mq2_re, mq2_im;      /* CPAIR: (p-k)-leg 1/(s + Mq2), Mq2 = conj   */
    double a, b, c;             /* DRESSED: (s + a)/(s^2 + b s + c), b^2 < 4c */
} orc_prop;

typedef struct {
    int dim;                    /* 3 or 4                                     */
    double mu2;                 /* subtraction point, real >= 0               */
    int n_radial, n_angular;    /* orders; n_radial % 4 == 0; n_angular >= 2,
                                   odd for tanh-sinh                          */
    double radial_scale;        /* L in |q| = L t/(1-t)                       */
    double detour_radius;       /* r of the half circle around a swept pole   */
    int angular_rule;           /* ORC_ANG_*                                  */
    int radial_rule;            /* ORC_RAD_*                                  */
} orc_params;

int orc_gauss_legendre(int n, double *x, double *w);
/* n nodes z_j = cos psi_j and weights w_j of the angular rule for
 * int_0^pi f(cos psi) sin^(D-2) psi dpsi = int_-1^1 f(z) (1-z^2)^((D-3)/2) dz */
int orc_angular_rule(int rule, int n, int dim, double *z, double *w);
/* x, G interleaved complex128 (re, im); kappa optional (may be NULL). */
int orc_eval_points(const orc_prop *P, const orc_params *Q, const double *x, long npts,
                    double *G, double *kappa, int nthreads);
int orc_grid_points(double re0, double re1, double im0, double im1, int m, int n, double *x);
/* Step 3 diagnostics (Sect. 5, Figs. 1-2). The angular integral of the
 * (p-k) leg as given, B(x, y) = int_0^pi sin^(D-2) psi [P2(s) - P2(y)] dpsi,
 * s = x + y - 2 sqrt(x y) cos psi, at one x and ny complex y (interleaved),
 * with Q's angular rule (or in closed form). */
int orc_angular_map(const orc_prop *P, const orc_params *Q, double xr, double xi,
                    const double *y, long ny, double *B);
/* Region 1 of Fig. 2: free[i] = 1 if no y on the positive real axis puts a
 * pole of the angular integrand on [0, pi] (the real-axis contour can be
 * kept), else 0. Found by scanning w = 4 x y/(x + y + M2)^2 along y > 0. */
int orc_region_map(const orc_prop *P, const double *x, long n, int *free_out);

#ifdef __cplusplus
}
#endif
#endif
