// Internal definitions shared by the host side of libgfc and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfc.h"

namespace gfc {

constexpr int kMaxRadial = 16384;
constexpr int kMaxAngular = 512;
constexpr int kMaxPairs = kMaxAngular / 2;
constexpr int kMaxRules = 32;
constexpr int kCounters = 16;  // per-call device counters (see gfc_capi.cpp)

// Contour of one pass of a point (Step 3, eq. 15).
enum PassKind : int { PASS_RAY = 0, PASS_DETOUR = 1 };

// What one launch evaluates.
enum LaunchMode : int {
    MODE_ALL = 0,        // every point (FP64 precision)
    MODE_BULK32 = 1,     // mixed, binary32: every point not in the binary64
                         // band; band points and points whose estimated
                         // rounding error exceeds mixed_rtol go to the list
    MODE_LIST64 = 2,     // mixed, binary64: the points of the list
    MODE_NODES = 3       // mixed: the node groups of the partially routed
                         // points (node_list), added to the bulk's G
};

// A partially routed point of the mixed precision: the binary32 bulk wrote
// the sum of its kept node groups; the groups in `mask` (bit g: the point's
// iterations [g gsz, (g + 1) gsz), an iteration being 32 consecutive nodes of
// a pass, numbered across the passes) are re-evaluated in the fallback
// arithmetic and added.
struct NodeEntry {
    int64_t point;
    unsigned mask;
    int gsz;
};
constexpr int kMaxGroups = 32;

// Per-propagator constants prepared on the host in FP64. Poles y_p are the
// zeros of the leg denominators in the y = q^2 plane.
struct PropConst {
    int kind;            // gfc_prop_kind
    // SCALAR
    double m2;
    // CPAIR after relabelling: yu = pole in the upper half plane, yl = conj(yu);
    // for Im x > 0 the k-leg carries yu (P1 = 1/(y - yu)) and the (p-k)-leg yl.
    double yu_re, yu_im;
    double arg_yu;       // in (0, pi)
    double yk0_re, yk0_im;   // k-leg pole as given (used on the real axis)
    // DRESSED: (s + a)/(s^2 + b s + c) = Rp/(s - yp) + Rm/(s - ym), ym = conj(yp)
    double a, b, c;
    double yp_re, yp_im, Rp_re, Rp_im;
    double arg_yp;       // in (0, pi)
    // binary64 band of the mixed precision
    double thr;          // branch point on the real axis: the cut is (-inf, thr]
    double pinch;        // |arg| of the ray direction where the angular
                         // integrand pinches (pi for real masses), < 0: none
};

// Kernel parameters (passed by value, __grid_constant__).
struct KParams {
    int dim;
    int n_r;             // radial nodes
    int n_s;             // nodes per detour segment (n_r / 4)
    int npair;           // angular pairs ((n_angular + 1) / 2; 0 with ang_exact)
    int mode;            // LaunchMode
    int ang_exact;       // angular integral in closed form (GFC_ANG_EXACT)
    // Omega1, delta, Re/Im of the dressed pole yp and residue Rp, as binary32
    // and as double-float (hi, lo) pairs, for the kernels of those arithmetics
    float f32c[6];
    float dfc[12];
    float om_df[2];      // Omega as a double-float (hi, lo) pair
    int use_grid;        // 1: x from the grid spec, 0: from x[]
    int64_t npts;
    // grid (Kernel 1)
    double re0, dre, im0, dim_im;
    int gm, gn;
    const double *x;     // interleaved complex128 (when !use_grid)
    double *G;           // interleaved complex128 output
    // node tables (device, FP64 and FP32 copies)
    const double2 *rad64;   // (rho_k, W_k)
    const double2 *rayp64;  // (rho_k^2, rho_k^(D-1) W_k): binary64 ray nodes from q = 0
    // double-float ray nodes from q = 0 in the frame of the ray, scaled by
    // sigma_k = 1/(1 + rho_k^2): [2k] = (rho_k^2 sigma_k, sigma_k),
    // [2k + 1] = (rho_k^(D-1) W_k sigma_k^3, 0), each a (hi, lo) pair
    const float4 *rayq_df;
    const float2 *rad32;
    const double2 *seg64;   // (t_k, w_k) on [0, 1]
    const float2 *seg32;
    const double2 *arc64;   // (cos pi t_k, sin pi t_k)
    const float2 *arc32;
    // double-float copies: (a.hi, a.lo, b.hi, b.lo) per node
    const float4 *rad_df, *seg_df, *arc_df;
    const double2 *tail64;  // n_r/2 nodes (rho, W) of the mapped half-line
    const float2 *tail32;   // (the clustered rule's last panel)
    const float4 *tail_df;
    int radial_rule;        // gfc_radial_rule
    double L, r_detour, K_D, mu2;
    double Omega, Omega1, delta;     // sum w, sum w t, 4 Omega1 - Omega (pairs)
    PropConst pc;
    // mixed-precision routing
    double cut_band, pinch_angle;
    double mixed_rtol;           // a-posteriori routing threshold (0: off)
    int64_t *list;               // points routed whole to the list arithmetic
    unsigned long long *list_count;
    // partial routing (one-shot calls; null in the server, whose routed
    // points go whole to `list`): node groups re-evaluated in the fallback
    NodeEntry *node_list;
    unsigned long long *node_list_count;
    float4 *snap;                // per warp slot [group][lane]: running sums at group ends
    int64_t snap_slots;          // warp slots of `snap`
    double *cond_out;            // optional per-point K_D sum_k M_k
    // compressed angular rules: Gauss rules of the discrete measure
    // sum_j e_j delta(t - t_j) with rule_n[r] nodes; rule r reproduces the full
    // pair sum of 1/(1 - w t) to rounding level when rho(w) >= rho_min{32,64}[r]
    int nrule;
    int rule_off[kMaxRules], rule_n[kMaxRules];
    // (the thresholds as sigma = (rho + 1/rho)/2, which the kernels compare)
    float sig_min32[kMaxRules], sig_min64[kMaxRules];
    // the same selection directly: rule r is exact to rounding for a node
    // when rule_n[r] >= K / ln(rho) (rho_min[r] = exp(K / rule_n[r])), with K
    // per arithmetic; rule_idx[m] is the first rule of at least m nodes
    // (nrule if none)
    float rule_k32, rule_k64;
    unsigned char rule_idx[128];
    const double *rules64;   // per node (tau, gamma, gamma tau)
    const float4 *rules32;   // per node (tau, gamma, gamma tau, 0)
    const float2 *rules_df;  // per node (tau, gamma, gamma tau) as double-float
    int rules_total;         // nodes over all rules
    // scratch
    const double *g0mu;  // complex G0(mu2) (2 doubles)
    unsigned long long *counter;  // work counter for dynamic point assignment
    unsigned long long *node_count;  // optional: contour nodes x angular nodes
    unsigned long long *pair_count;  // optional: angular pairs actually evaluated
    unsigned long long *pair_full_count;  // optional: the part of them over the full table
};

// Angular pair table: t = cos^2 psi_j, e = w t^2, g = w t^3 (w includes the
// sin^(D-2) psi weight), for the pairs (psi_j, pi - psi_j), j < npair.
template <typename T, int NP>
struct AngTab {
    T t[NP], e[NP], g[NP];
};

// size of the constant-bank table of a kernel specialised for NP pairs
// (NP = 0: any number of pairs, table read from shared memory)
template <int NP>
constexpr int tab_size() { return NP > 0 ? NP : 1; }

// Host-side launchers (gfc_kernels.cu). Tables: (t, e, g) per pair, FP64.
struct DevTables {
    const double *ang64;     // 3 * npair, interleaved (t, e, g)
    const float *ang32;
    const float2 *ang_df;    // double-float copy
    const double *t, *e, *g; // host copies
};

// Continuous batching: one work item is a contiguous point range of one
// request slot.
struct BatchItem {
    int slot;
    int pad;
    int64_t p0, p1;
};

struct BatchLaunch {
    const KParams *slots;        // device array of request descriptors
    const BatchItem *items;      // device
    const int64_t *offs;         // device, first launch-wide index of item i
    int nitems;
    int64_t total;               // points in the launch
    unsigned long long *counter; // device, zero before the launch
    int mode;
    int npair;
    int rules_total;             // compressed-rule nodes of the launch's angular rule
    int radial_rule;             // gfc_radial_rule shared by the launch's requests
    int ang_exact;               // closed-form angle, shared likewise
};

cudaError_t launch_batch(const BatchLaunch &bl, const DevTables &tb, int arith, bool two_terms,
                         cudaStream_t st);
cudaError_t launch_g0mu(const KParams &kp, const DevTables &tb, double mu2, double *partials,
                        int nwarps, unsigned *ticket, double *g0mu_out,
                        unsigned long long *counters, cudaStream_t st);
// arithmetic of a launch
enum Arith : int { ARITH_F64 = 0, ARITH_F32 = 1, ARITH_DF = 2 };
cudaError_t launch_eval(const KParams &kp, const DevTables &tb, int arith, cudaStream_t st);
cudaError_t launch_grid_points(double re0, double dre, double im0, double dim_im, int m, int n,
                               double *x, cudaStream_t st);

// ---------------------------------------------------------------------------
// host side (gfc_capi.cpp), shared with the serving runtime
// ---------------------------------------------------------------------------
struct Tables;
int fail(int code, const char *msg);
// Device allocations of the library go through these: they honour the test
// hook gfc_test_fail_allocations (the next n allocations report
// cudaErrorMemoryAllocation without calling the runtime).
cudaError_t dev_malloc(void **p, size_t bytes);
cudaError_t dev_malloc_async(void **p, size_t bytes, cudaStream_t s);
// Test hooks: an evaluation launch (one-shot or batched) that reports
// cudaErrorLaunchOutOfResources without launching (gfc_test_fail_launches),
// and the full angular table in place of the compressed rules
// (gfc_test_full_angular_rule).
bool take_injected_launch_failure();
bool full_rule_forced();
int cuda_fail(cudaError_t e, const char *what);
int check_params_c(const void *params);
int check_grid_c(const void *grid);
int make_prop_c(const void *prop, const void *params, PropConst &pc);
// angular pairs of a parameter set (0 when the angular integral is exact)
inline int npair_of(const gfc_params *p)
{
    return p->angular_rule == GFC_ANG_EXACT ? 0 : (p->n_angular + 1) / 2;
}

int get_tables_c(int dev, int n_r, int n_a, int dim, double L, int ang_rule, Tables **out,
                 size_t *bytes);
void fill_kparams_c(KParams &kp, const void *params, const Tables &T, const PropConst &pc);
DevTables dev_tables_c(const Tables &T);

}  // namespace gfc
