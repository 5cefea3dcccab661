/*
 * gfc.h — C ABI of the GB300 library that evaluates Taylor-subtracted
 * two-point correlators on grids of complex external momentum p^2 = x.
 *
 * The operation (Windisch, Alkofer, Haase, Liebmann, arXiv:1205.0752):
 *
 *   G(x) = G0(x) - G0(mu2),
 *   G0(x) = K_D int_C dy (1/2) y^((D-2)/2) int_0^pi dpsi sin^(D-2) psi
 *              P1(y) [ P2(x + y - 2 sqrt(x y) cos psi) - P2(y) ]
 *
 * Sect. 2 Step 1 (eqs. 5-11: hyperspherical reduction, K_D = S_(D-2)/(2 pi)^D),
 * Step 2 (eqs. 12-14, 20: BPHZ subtraction (1 - t^0) at x = 0), Step 3 (eq. 15:
 * radial contour C deformed around the poles and the angular cut, Sect. 5.3),
 * Steps 4-5 (Sect. 4, Kernels 1 and 2: a homogeneous M x N grid of x and one
 * 2-D Gauss-Legendre quadrature per point). The physical normalisation is
 * int d^Dq / (2 pi)^D; 16 pi^2 G is the paper's rescaled eq. 18 for its
 * worked example.
 *
 * Conventions for every call:
 *  - the return value is a status: GFC_OK (0) or a negative GFC_E* code;
 *    gfc_last_error() gives a thread-local message for the last failure;
 *  - no C++ exception crosses this boundary;
 *  - complex arrays are interleaved complex128: element k is (re, im) at
 *    [2k, 2k+1], 16-byte aligned;
 *  - "device" pointers are CUDA global-memory pointers on the current device;
 *    the caller owns them and keeps them alive until the work on `stream`
 *    (a cudaStream_t passed as void*; NULL = the legacy default stream) has
 *    finished; the calls return once the work is enqueued;
 *  - on an invalid argument nothing is enqueued and no output is written;
 *  - the library owns its node tables and scratch (device memory it
 *    allocates on first use per device and keeps until gfc_release()).
 */
#ifndef GFC_H
#define GFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GFC_VERSION_MAJOR 1
#define GFC_VERSION_MINOR 6

enum {
    GFC_OK = 0,
    GFC_EINVAL = -1,     /* an argument is out of range; nothing was done      */
    GFC_ENOMEM = -2,     /* device or host allocation failed                   */
    GFC_EBUDGET = -3,    /* a request does not fit the server's memory budget   */
    GFC_ECUDA = -4,      /* a CUDA runtime call failed (message has the name)  */
    GFC_ETIMEOUT = -5,   /* a wait ran out of time                             */
    GFC_ECANCELED = -6,  /* the request was cancelled                          */
    GFC_EBUSY = -7,      /* the server is shutting down or the queue is full   */
    GFC_ENOTFOUND = -8   /* unknown ticket                                     */
};

/* Propagator on both legs (Sect. 5, eq. 16; the dressed form is the
 * propagator family of the correlators studied in ref. [aw3] of the paper). */
typedef enum {
    GFC_PROP_SCALAR = 0,   /* 1/(s + m2), m2 > 0 real, on both legs            */
    GFC_PROP_CPAIR = 1,    /* k-leg 1/(s + Mk2), (p-k)-leg 1/(s + Mq2),
                              Mq2 = conj(Mk2), Im Mk2 != 0; the paper's example
                              is Mk2 = +i/2, Mq2 = -i/2 (eq. 19)               */
    GFC_PROP_DRESSED = 2   /* (s + a)/(s^2 + b s + c) on both legs, b^2 < 4c   */
} gfc_prop_kind;

typedef struct {
    int kind;                   /* gfc_prop_kind                               */
    double m2;                  /* SCALAR                                      */
    double mk2_re, mk2_im;      /* CPAIR                                       */
    double mq2_re, mq2_im;      /* CPAIR                                       */
    double a, b, c;             /* DRESSED                                     */
} gfc_propagator;

typedef enum {
    GFC_FP64 = 0,    /* every step in IEEE binary64                            */
    GFC_MIXED = 1,   /* angular sums and per-node set-up in binary32 with
                        compensated binary32 radial sums, binary64 for the
                        epilogue; the points of the cut band whole in
                        binary64; a point whose estimated binary32 error is
                        above mixed_rtol |G| has the node groups with the
                        largest share of that estimate evaluated again in the
                        mixed_fallback arithmetic (all of its nodes next to
                        an angular pinch)                                    */
    GFC_F32X2 = 2    /* every step in double-float arithmetic (a value is the
                        sum of two binary32 numbers, ~48 bits) on the binary32
                        pipes; same tolerance target as GFC_FP64               */
} gfc_precision;

/* Angular rule for int_0^pi f(cos psi) sin^(D-2) psi dpsi (Sect. 4 of the
 * paper: the angular integral by tanh-sinh quadrature in z = cos psi, with
 * Gauss-Chebyshev rules of the first and second kind as a check). */
typedef enum {
    GFC_ANG_GAUSS_LEGENDRE = 0,  /* Gauss-Legendre in psi on [0, pi] (default) */
    GFC_ANG_TANH_SINH = 1,       /* tanh-sinh in z with weight (1-z^2)^((D-3)/2):
                                    z = tanh(pi/2 sinh(k h)), k = -N..N,
                                    n_angular = 2N + 1 (odd), h = 3/N          */
    GFC_ANG_CHEBYSHEV1 = 2,      /* psi_j = (j - 1/2) pi/n, weight
                                    (pi/n) sin^(D-2) psi_j                     */
    GFC_ANG_CHEBYSHEV2 = 3,      /* psi_j = j pi/(n + 1), weight
                                    pi/(n+1) sin^(D-2) psi_j (Gaussian for D=4) */
    GFC_ANG_EXACT = 4            /* the angular integral in closed form, the
                                    limit n -> infinity of every rule above:
                                    no quadrature error in psi, which dominates
                                    next to the negative real axis;
                                    n_angular is ignored                       */
} gfc_angular_rule;

/* Radial rule of the rays that start at q = 0 (Step 3; the paper uses
 * Gauss-Legendre and notes that contours close to singular structures need
 * many nodes, Sect. 4). */
typedef enum {
    GFC_RAD_MAPPED = 0,     /* n_radial Gauss-Legendre nodes on |q| = L t/(1-t)
                               (default)                                       */
    GFC_RAD_CLUSTERED = 1   /* when a pole +-sqrt(y_p) of the propagator lies
                               within ~37 degrees of the ray (distance d below
                               0.75 of its projection c on the ray): n_radial/4
                               nodes on each of [0, c] and [c, 2c], mapped by
                               |q| = c + d sinh(s), then n_radial/2 on the
                               mapped half-line from 2c; else as MAPPED. With
                               GFC_ANG_EXACT this resolves the points next to
                               the negative real axis beyond threshold.       */
} gfc_radial_rule;

typedef struct {
    int dim;               /* 3 or 4                                           */
    double mu2;            /* subtraction point, real, >= 0; G(mu2) = 0        */
    int n_radial;          /* Gauss-Legendre order on the radial half-line;
                              multiple of 4, 4 <= n_radial <= 16384            */
    int n_angular;         /* order of the angular rule, 2 <= n_angular <= 512;
                              odd for tanh-sinh (an odd order puts a node at
                              psi = pi/2)                                     */
    double radial_scale;   /* L in |q| = L t/(1-t); > 0                        */
    double detour_radius;  /* r of the half circle around a k-leg pole; > 0 and
                              below half the pole's modulus (paper: 0.1)       */
    int precision;         /* gfc_precision                                    */
    double cut_band;       /* MIXED: points closer than this to a branch cut
                              half-line are evaluated whole in binary64 (0.05) */
    double pinch_angle;    /* MIXED: points whose radial ray lies within this
                              angle (radians) of a leg's pinch direction are
                              evaluated whole in binary64 (default 0: off)     */
    double mixed_rtol;     /* MIXED: a point whose binary32 sum has an
                              estimated rounding error above mixed_rtol |G|
                              has its node groups (a group: gsz x 32
                              consecutive radial nodes, at most 32 groups per
                              point) with the largest share of the estimate
                              evaluated again in the mixed_fallback
                              arithmetic, until the estimate of the groups
                              kept in binary32 is below mixed_rtol |G| / 4
                              (default 1e-6; 0 turns this off, leaving the cut
                              band only). The serving runtime evaluates such
                              points whole in the mixed_fallback arithmetic. */
    int mixed_fallback;    /* MIXED: arithmetic of what is evaluated again:
                              GFC_F32X2 (default: double-float, ~48 bits,
                              about 5x the GB300's FP64 rate) or GFC_FP64     */
    int angular_rule;      /* gfc_angular_rule (default Gauss-Legendre)        */
    int radial_rule;       /* gfc_radial_rule (default mapped half-line)       */
} gfc_params;

/* Cell-centred grid of Kernel 1 (Sect. 4): x_ij = re0 + (i + 1/2)(re1-re0)/m
 * + i (im0 + (j + 1/2)(im1-im0)/n), i < m along Re x, j < n along Im x,
 * stored at flat index i*n + j. */
typedef struct {
    double re0, re1, im0, im1;
    int m, n;
} gfc_grid;

/* Per-call counters of the last evaluation on this thread. */
typedef struct {
    int64_t points;            /* points of the call                           */
    int64_t points_fp64;       /* MIXED: points evaluated whole in binary64
                                  (the cut band, points next to a pinch);
                                  FP64: all                                    */
    int64_t node_evals;        /* sum over evaluated points of contour nodes x
                                  angular nodes (all passes; binary32 and
                                  binary64 evaluations both counted)            */
    int kernel_launches;       /* kernels enqueued by the call                  */
    int64_t pairs_evaluated;   /* angular +-psi pairs the kernels evaluated; the
                                  compressed angular rules make this smaller
                                  than node_evals / 2 at the same result        */
    int64_t node_evals_fallback;  /* MIXED: the part of node_evals evaluated by
                                  the fallback arithmetic (the re-evaluated
                                  node groups of routed points); else 0         */
    int64_t pairs_fallback;    /* MIXED: the part of pairs_evaluated evaluated
                                  by the fallback arithmetic; else 0            */
    int64_t pairs_full_table;  /* the part of pairs_evaluated summed over the
                                  full angular table (nodes next to a pinch,
                                  where no compressed rule is exact)            */
    int64_t pairs_full_table_fallback;  /* MIXED: the fallback's part of it     */
    int64_t points_partial;    /* MIXED: routed points whose worst node groups
                                  were re-evaluated in the fallback arithmetic  */
    int64_t node_evals_list64; /* MIXED: node evaluations of the points
                                  evaluated whole in binary64                   */
    int64_t pairs_list64;      /* MIXED: their angular pairs                    */
    int64_t pairs_full_table_list64;  /* MIXED: the full-table part of those    */
} gfc_eval_stats;

const char *gfc_strerror(int status);
/* Thread-local text of the last failure on this thread ("" if none). */
const char *gfc_last_error(void);
int gfc_version(int *major, int *minor);

/* Defaults: D = 4, mu2 = 1, 2048 x 256 nodes, L = 1, r = 0.1, FP64,
 * cut_band 0.05, pinch_angle 0, mixed_rtol 1e-6, mixed_fallback F32X2,
 * angular_rule Gauss-Legendre, radial_rule mapped. */
int gfc_params_default(gfc_params *p);

/* Steps 4-5 on caller-given points: x and G are DEVICE arrays of npts
 * complex128. A point on the negative real axis (Im x = 0, Re x < 0) lies on
 * the cut side where the method is undefined; its G is written as NaN.
 * npts = 0 is valid and enqueues nothing. */
int gfc_eval_points(const gfc_propagator *prop, const gfc_params *params,
                    const double *x, int64_t npts, double *G, void *stream);

/* As gfc_eval_points, and if `cond` is not NULL it receives, per point, the
 * rounding-error scale K_D (sqrt(sum_k (M_k kappa_k)^2) + sum_k M_k) (DEVICE
 * array of npts doubles), where M_k is the magnitude of node k's contribution
 * and kappa_k its relative condition number: |y|/|y + M2| per propagator
 * factor, (|x| + |y|)/|a| for the angular denominator and, in binary32
 * (GFC_MIXED), |w|/min_j |1 - w t_j| for the angular sum. The rounding error
 * of a point is a small multiple of the unit roundoff of its precision times
 * this number. Double-float computes no scale and writes 0 for every point
 * under GFC_F32X2. Under GFC_MIXED the scale is that of the part of the sum
 * kept in binary32 (the whole point, or the kept node groups of a point whose
 * other groups the fallback evaluated again; 0 where nothing is kept, next
 * to an angular pinch), and the binary64 scale for the cut band, evaluated
 * whole in binary64. 0 is also written where nothing is summed (the cut side,
 * x = mu2). */
int gfc_eval_points_cond(const gfc_propagator *prop, const gfc_params *params,
                         const double *x, int64_t npts, double *G, double *cond, void *stream);

/* Steps 4-5 on the cell-centred grid (Kernel 1 fused into Kernel 2): G is a
 * DEVICE array of m*n complex128, G[i*n + j]. GFC_EINVAL if a grid row lies
 * on the negative real axis. */
int gfc_eval_grid(const gfc_propagator *prop, const gfc_params *params,
                  const gfc_grid *grid, double *G, void *stream);

/* Kernel 1 alone (Step 4): writes the m*n grid points to the DEVICE array x. */
int gfc_grid_points(const gfc_grid *grid, double *x, void *stream);

/* End-to-end form of gfc_eval_points for HOST arrays (pageable or pinned):
 * copies x to the device, evaluates, copies G back and waits for the stream;
 * uses library-owned device buffers. */
int gfc_eval_points_host(const gfc_propagator *prop, const gfc_params *params,
                         const double *x_host, int64_t npts, double *G_host, void *stream);

/* gfc_eval_points (GFC_FP64 only) for callers that cannot allocate device
 * memory: code that runs while another component owns the device heap (a
 * framework's caching allocator, an embedding with a fixed device-memory
 * plan), or code that must not pay for the device-wide synchronisation that
 * cudaFree (and often cudaMalloc) implies. The paper has no counterpart.
 * Its node tables and scratch live in one file-scope device array of about
 * 170 KB, so the call allocates nothing (no cudaMalloc, cudaFree or
 * allocating library call); x and G are the caller's DEVICE arrays as for
 * gfc_eval_points. Limits: precision GFC_FP64, n_radial <= 4096, even
 * n_angular <= 512, the Gauss-Legendre angular rule and the mapped radial
 * rule, and the full angular table (no compressed rules); anything else
 * gives GFC_EINVAL. The tables are uploaded from static host arrays of the
 * library with cudaMemcpyAsync from pageable memory, which may wait for the
 * work already queued on `stream`. The array is shared by every call on a
 * device and keeps the last call's contents: calls that overlap on the GPU
 * (other streams or host threads) race on it. The first call on a device
 * looks up the array's address with that device current; make that first
 * call before any stream capture. */
int gfc_eval_points_noalloc(const gfc_propagator *prop, const gfc_params *params,
                            const double *x, int64_t npts, double *G, void *stream);

/* Step 3 diagnostics (Sect. 5, Figs. 1-2), binary64.
 *
 * gfc_angular_map: the angular integral of the (p-k) leg as given (no
 * relabelling), B(x, y) = int_0^pi sin^(D-2) psi [P2(s) - P2(y)] dpsi with
 * s = x + y - 2 sqrt(x) sqrt(y) cos psi, at one external x = x_re + i x_im
 * and ny complex y (DEVICE arrays of complex128, y in, B out), with the
 * params' angular rule (or in closed form, GFC_ANG_EXACT). Evaluated over a
 * grid of y it is the density plot of Fig. 1: B jumps across the branch cut
 * of eq. 25; a y on a node of the rule's pole set gives inf/NaN. Uses dim,
 * n_angular and angular_rule of params (the radial fields are validated but
 * unused). GFC_EINVAL for bad params or pointers. */
int gfc_angular_map(const gfc_propagator *prop, const gfc_params *params, double x_re,
                    double x_im, const double *y, int64_t ny, double *B, void *stream);

/* Test hook (host-side fault injection; the paper has no counterpart): the
 * next n device allocations the library makes -- node tables, per-stream
 * scratch, mixed-precision lists, host-path staging, serving buffers -- fail
 * as if the runtime had reported cudaErrorMemoryAllocation, so that error
 * paths can be exercised without faulting a GPU. The failing call returns
 * GFC_ECUDA with the failure in gfc_last_error(); n = 0 clears the hook.
 * GFC_EINVAL for n < 0. */
int gfc_test_fail_allocations(int n);

/* Test hook (host-side fault injection; the paper has no counterpart): the
 * next n evaluation-kernel launches (Kernel 2, one-shot or batched by the
 * server; not the G0(mu2) kernel) report cudaErrorLaunchOutOfResources
 * without launching anything, so that the error paths of the one-shot calls
 * and of the serving loop can be exercised without faulting a GPU. A one-shot
 * call then returns GFC_ECUDA; a served request carried by such a launch
 * finishes with GFC_ECUDA and its output is not written. n = 0 clears the
 * hook. GFC_EINVAL for n < 0. */
int gfc_test_fail_launches(int n);

/* Test switch (the paper has no counterpart): on != 0 makes every later
 * evaluation sum each radial node's angular integral over the full angular
 * table instead of the smallest compressed Gauss rule of the table's discrete
 * measure that reproduces that sum to rounding level; on = 0 restores the
 * compressed rules. Process-wide; takes effect for calls (and server
 * admissions) made after it returns. Used to show, at full size, that the
 * two give the same results. Always GFC_OK. */
int gfc_test_full_angular_rule(int on);

/* Test hook (host only, no device work): the angular tables the evaluation
 * kernels use for n_angular nodes of angular_rule in dimension dim (the
 * integrand's angular part of eq. 20 summed over the +-psi pairs of a
 * symmetric rule, Sect. 4). *npair receives the pair count np and, if pairs
 * is not NULL, pairs[3j .. 3j+2] = (t_j, e_j, g_j) with t_j = cos^2 psi_j,
 * e_j = w_j t_j^2, g_j = e_j t_j (np <= max_pairs). *nrule receives the
 * number of compressed rules (at most 32): Gauss rules of the discrete
 * measure sum_j e_j delta(t - t_j), rule r with rule_n[r] nodes, used by a
 * binary64 or double-float node whose Bernstein-ellipse parameter of the pole
 * 1/w is at least rho_min[r]; if rules is not NULL it receives their nodes in
 * order, 3 doubles (tau, gamma, gamma tau) each (sum of rule_n <=
 * max_rule_nodes). rule_n and rho_min may be NULL. GFC_EINVAL for parameters
 * gfc_eval_points would reject, NULL npair or nrule, or short capacity. */
int gfc_test_angular_rules(int n_angular, int dim, int angular_rule, double *pairs, int max_pairs,
                           int *npair, double *rules, int max_rule_nodes, int *rule_n,
                           float *rho_min, int *nrule);

/* gfc_region_map: region 1 of Fig. 2. For each of npts external x (DEVICE
 * complex128), free_out[i] (DEVICE int32) = 1 if the branch cut of B(x, .)
 * -- the curve y = (sqrt(x) cos th +- sqrt(-x sin^2 th - M2))^2, th in
 * [0, pi], of eqs. 24-25 for each pole s = -M2 of the (p-k) leg as given --
 * does not cross the positive real y-axis, so the original contour along it
 * can be kept; else 0. The curve is traced on 4096 samples of th, so points
 * within about that resolution of the region's boundary may go either way. */
int gfc_region_map(const gfc_propagator *prop, const double *x, int64_t npts,
                   int32_t *free_out, void *stream);

/* Counters of the last gfc_eval_* call made on this thread; waits for the
 * work of that call to finish (the counts are read from the device). */
int gfc_last_stats(gfc_eval_stats *out);

/* Measurement support (the paper has no counterpart): the throughput of the
 * scalar pipes that bound the evaluation kernels, measured on the current
 * device. Each rate is thread operations per second of a microkernel that
 * runs 8 or 16 independent dependency chains per thread on SMs x 4 or 8
 * blocks of 256 threads (the best of these configurations, each the best of
 * two timed launches of about seconds/4 after a calibration run, CUDA events
 * on `stream`): binary64 FMA (plain chains, and chains interleaved with an
 * independent binary32 FMA chain), multiply and add (the FP64 pipe), binary32 FMA
 * (the FMA pipe) and rcp.approx.ftz.f32 (the special-function unit). These
 * are the denominators of the kernels' executed-work fractions. Blocks until
 * the probes have finished (about 10 x seconds). GFC_EINVAL for out = NULL or
 * seconds outside (0, 10]. */
typedef struct {
    double dfma_per_s;     /* binary64 fused multiply-adds per second          */
    double dmul_per_s;     /* binary64 multiplies per second                   */
    double dadd_per_s;     /* binary64 adds per second                         */
    double ffma_per_s;     /* binary32 fused multiply-adds per second          */
    double rcp32_per_s;    /* binary32 approximate reciprocals per second      */
    int sm_count;          /* multiprocessors of the device                    */
    double dfma_mhz;       /* SM clock during the best binary64 FMA launch
                              (clock64 over the global timer on one SM)        */
    double ffma_mhz;       /* the same for the binary32 FMA launch             */
    double fp64_mix_per_s; /* binary64 FMA, multiply and add in the proportions
                              5 : 2 : 1 of the binary64 evaluation kernel, FP64
                              instructions per second (the FP64 pipe issues a
                              mixed stream faster than one operation alone)   */
} gfc_pipe_peaks;
int gfc_measure_pipe_peaks(gfc_pipe_peaks *out, double seconds, void *stream);

/* Frees the library-owned device memory of the current device (node tables,
 * scratch, staging buffers). Must not overlap any work still running. */
int gfc_release(void);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of grid requests into persistent launches.   */
/* ------------------------------------------------------------------------ */

typedef struct gfc_server gfc_server;

typedef struct {
    uint64_t submitted, completed, rejected, canceled;
    double p50_ms, p99_ms;          /* submit -> completion latency           */
    double points_per_s;            /* completed points / wall time since create */
    int64_t points_done;
    size_t bytes_in_use, bytes_budget;
    int64_t launches;               /* batched launches so far                */
    int queued, active;             /* requests waiting / on the device       */
} gfc_stats;

/* One server per device; `hbm_budget_bytes` bounds the device memory the
 * server holds for admitted requests (output grids and staging); at most
 * `max_slots` requests are on the device at once. */
int gfc_server_create(int device, size_t hbm_budget_bytes, int max_slots, gfc_server **out);

/* Queues one grid request and returns at once with a ticket. G_host receives
 * m*n complex128 values, G[i*n + j]; it stays valid until the request
 * finishes (gfc_server_wait or poll report it done). It is either host memory
 * (pageable or pinned: the server copies the grid into it through its own
 * pinned staging once every launch of the request has finished) or device
 * memory of the server's device (the kernels write it in place, and the
 * server holds no output buffer for the request). GFC_EBUDGET if the request
 * alone exceeds the budget, GFC_EINVAL on a bad argument (device memory of
 * another device included), GFC_EBUSY when shutting down. A request whose
 * launches or copies hit a CUDA error finishes with GFC_ECUDA and no result
 * (its host array is not written). */
int gfc_server_submit(gfc_server *s, const gfc_propagator *prop, const gfc_params *params,
                      const gfc_grid *grid, double *G_host, uint64_t *ticket);

/* done = 1 once the request finished; status then holds its result code. */
int gfc_server_poll(gfc_server *s, uint64_t ticket, int *done, int *status);

/* Waits up to timeout_ms (< 0: without limit) for the request; returns its
 * status, or GFC_ETIMEOUT if it is still running when the time is up. */
int gfc_server_wait(gfc_server *s, uint64_t ticket, int timeout_ms);

/* Cancels a request that has not finished: no further launch carries its
 * work. A host G_host is not written after this returns GFC_OK; a device
 * G_host may still be written by a launch already in flight until
 * gfc_server_wait reports GFC_ECANCELED. */
int gfc_server_cancel(gfc_server *s, uint64_t ticket);

int gfc_server_stats(gfc_server *s, gfc_stats *out);

/* One request's record, for per-request logs (any time after submission). */
typedef struct {
    int status;               /* final status; GFC_ETIMEOUT while not finished  */
    int state;                /* 0 queued, 1 on the device, 2 finished          */
    int64_t points;           /* points of the grid                             */
    int64_t points_routed;    /* MIXED: points re-evaluated by the fallback
                                 arithmetic; -1 if not (yet) known              */
    double queue_ms;          /* submission -> admission; -1 while queued       */
    double total_ms;          /* submission -> completion; -1 while running     */
    int64_t launches;         /* batched launches that carried its work         */
    size_t bytes;             /* device bytes admitted for it                   */
} gfc_request_info;

/* GFC_ENOTFOUND for an unknown ticket. */
int gfc_server_request_info(gfc_server *s, uint64_t ticket, gfc_request_info *out);

/* Estimated work the server has not launched yet (queued and admitted
 * requests), in its scheduling units (binary32 angular pair evaluations; a
 * binary64 pair counts 24, a double-float pair 6). */
int gfc_server_load(gfc_server *s, double *work);

/* Cancels what is still queued, drains what is on the device, frees all. */
int gfc_server_destroy(gfc_server *s);

/* ------------------------------------------------------------------------ */
/* Several devices: one server per device, each request handed whole to the  */
/* server with the least estimated work outstanding. Every grid point is     */
/* independent (Sect. 1), so a request needs nothing from the other devices. */
/* ------------------------------------------------------------------------ */

typedef struct gfc_router gfc_router;

/* One server per entry of devices[0..ndevices) (1 <= ndevices <= 256; an
 * entry may repeat), each with the given budget and slots as for
 * gfc_server_create. */
int gfc_router_create(const int *devices, int ndevices, size_t hbm_budget_bytes, int max_slots,
                      gfc_router **out);

/* As gfc_server_submit, on the least-loaded server (gfc_server_load; ties go
 * to the lowest index). G_host is host memory, or device memory of the
 * device that the chosen server runs on (GFC_EINVAL if it belongs to another
 * device). The ticket names the server in its low 8 bits. */
int gfc_router_submit(gfc_router *r, const gfc_propagator *prop, const gfc_params *params,
                      const gfc_grid *grid, double *G_host, uint64_t *ticket);
int gfc_router_poll(gfc_router *r, uint64_t ticket, int *done, int *status);
int gfc_router_wait(gfc_router *r, uint64_t ticket, int timeout_ms);
int gfc_router_cancel(gfc_router *r, uint64_t ticket);

/* The index-th server (for gfc_server_stats, gfc_server_load), and the server
 * index and server ticket that a router ticket names (for
 * gfc_server_request_info). */
int gfc_router_server(gfc_router *r, int index, gfc_server **out);
int gfc_router_server_of(gfc_router *r, uint64_t ticket, int *index, uint64_t *server_ticket);

/* Destroys every server (gfc_server_destroy) and the router. */
int gfc_router_destroy(gfc_router *r);

#ifdef __cplusplus
}
#endif
#endif /* GFC_H */
