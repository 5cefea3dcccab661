// Serving runtime of libgfc: continuous batching of grid requests.
//
// A scheduler thread admits queued requests into device slots while the
// server's memory budget and slot count allow, computes each admitted
// request's G0(mu2) on the device, then carves the requests' points into work
// items and issues persistent batched launches (eval_batch_kernel). One launch
// mixes items of the active requests that share its kernel variant
// (binary32/binary64, angular order, dimension, number of terms, launch
// mode); variants run on separate streams, so requests of different kinds
// overlap on the device. Admission and launch composition are cost-aware:
// requests are served least estimated remaining work first, aged by their
// waiting time so that none starves. Each launch is sized to a bounded amount
// of work and only a few are on the device at once, so a request that
// arrives while others run joins the next launches, on a high-priority stream
// when it is short. When all items of a request have finished, its grid is
// copied to the host through a pinned staging buffer (or was written in
// place, for device outputs), its slot and memory are freed, and its latency
// (submit to completion) is recorded.
#include <cuda_runtime.h>

#include <algorithm>

#include <nvtx3/nvToolsExt.h>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "gfc.h"
#include "gfc_internal.h"

namespace gfc {

int check_grid_c(const void *grid);

namespace {

using clk = std::chrono::steady_clock;

constexpr int kStreams = 4;          // launch streams: 0, 1 high priority; 2, 3 low
constexpr int kRing = 16;            // launch records
constexpr int kMaxInflight = 6;      // launches queued or running on the device at once
constexpr int kMaxItems = 4096;      // work items per launch
constexpr int kG0Warps = 512;
// work per launch in units of binary32 pair evaluations (about 10-20 ms)
constexpr double kLaunchWork = 7.5e10;
// ageing of the scheduling key: half the work units the device completes per
// second, so that a request that has waited t seconds ranks as if it had the
// work the device does in t/2 seconds less left. (A queueing model of the
// serving mix's measured request costs at 70 % load: ageing at the full
// device rate raises p50 and p99 by 10-40 % against half of it; no ageing
// at all starves the largest requests.)
constexpr double kAgeRate = 0.5 * kLaunchWork / 0.015;
// fraction of a mixed request's points that its fallback is expected to
// re-evaluate (the key's estimate until the count is known)
constexpr double kMixedRouted = 0.45;
constexpr double kFp64Weight = 24.0; // binary64 pair cost in binary32 pair units
constexpr double kDfWeight = 6.0;    // double-float pair cost in binary32 pair units

enum ReqState { R_QUEUED, R_ACTIVE, R_COPYING, R_DONE };

struct Phase {
    int mode;          // LaunchMode
    int arith;         // Arith
    int64_t next;      // first point (or list entry) not yet put in an item
    int64_t end;       // points (or list entries) of the phase; -1: not known yet
    int64_t items_out; // items launched and not finished
};

struct Request {
    uint64_t ticket = 0;
    gfc_propagator prop{};
    gfc_params params{};
    gfc_grid grid{};
    double *G_host = nullptr;           // caller's output (host or device)
    bool G_on_device = false;           // G_host is device memory of the server's device
    int64_t npts = 0;
    size_t bytes = 0;
    ReqState state = R_QUEUED;
    int status = GFC_OK;
    int slot = -1;
    double *G_dev = nullptr;
    Tables *T = nullptr;
    KParams kp{};
    std::vector<Phase> phases;
    int64_t *list_dev = nullptr;        // binary64 list (mixed precision)
    bool count_pending = false;         // list length being read back
    cudaEvent_t count_done = nullptr;
    bool canceled = false;
    bool failed = false;                // a CUDA call on its behalf failed
    std::string fail_msg;
    void *pinned = nullptr;
    size_t pinned_size = 0;
    cudaEvent_t copy_done = nullptr;
    double work_left = 0.0;             // estimated work not yet launched (units of kLaunchWork)
    clk::time_point t_submit, t_admit, t_done;
    bool admitted = false;
    int64_t launches = 0;               // batched launches that carried its work
    int64_t routed = -1;                // MIXED: points re-evaluated by the fallback
};

struct LaunchRec {
    cudaEvent_t done = nullptr;
    bool busy = false;
    bool failed = false;                // a call issuing the launch failed
    std::string fail_msg;
    std::vector<std::tuple<Request *, int, int64_t>> reqs;   // request, phase, items
    BatchItem *items_dev = nullptr;
    int64_t *offs_dev = nullptr;
    unsigned long long *counter_dev = nullptr;
    BatchItem *items_host = nullptr;    // pinned
    int64_t *offs_host = nullptr;       // pinned
};

// arith, npair, dim, two terms, mode, angular rule, radial rule: the requests
// of one launch share its angular tables and its kernel
using GroupKey = std::tuple<int, int, int, int, int, int, int>;

}  // namespace

}  // namespace gfc

struct gfc_server {
    int device = 0;
    size_t budget = 0;
    int max_slots = 0;
    std::mutex mu;
    std::condition_variable cv_done, cv_work;
    std::thread th;
    bool stopping = false;
    uint64_t next_ticket = 1;
    std::map<uint64_t, std::unique_ptr<gfc::Request>> reqs;
    std::deque<gfc::Request *> queue;
    std::vector<gfc::Request *> active;
    std::vector<int> free_slots;
    size_t bytes_in_use = 0;
    size_t table_bytes = 0;
    // device state
    cudaStream_t admit_stream = nullptr, copy_stream = nullptr;
    cudaStream_t streams[gfc::kStreams] = {};
    cudaEvent_t admit_event = nullptr;
    gfc::KParams *slots_dev = nullptr;
    gfc::KParams *slots_host = nullptr;   // pinned mirror
    double *g0mu_dev = nullptr;
    unsigned long long *slot_counts_dev = nullptr;   // list length per slot
    unsigned long long *slot_counts_host = nullptr;  // pinned
    double *partials_dev = nullptr;
    unsigned *ticket_dev = nullptr;
    unsigned long long *dummy_counters = nullptr;
    gfc::LaunchRec ring[gfc::kRing];
    int next_stream = 0;
    // pinned host staging pool
    std::vector<std::pair<void *, size_t>> pinned_free;
    // statistics
    uint64_t n_submitted = 0, n_completed = 0, n_rejected = 0, n_canceled = 0;
    int64_t points_done = 0, launches = 0;
    std::vector<double> lat_ms;
    std::chrono::steady_clock::time_point t_first, t_last;
    bool any_done = false;
    int error = GFC_OK;
};

namespace gfc {
namespace {

void *pinned_get(gfc_server *s, size_t n)
{
    size_t best = (size_t)-1;
    int bi = -1;
    for (int i = 0; i < (int)s->pinned_free.size(); ++i)
        if (s->pinned_free[i].second >= n && s->pinned_free[i].second < best) {
            best = s->pinned_free[i].second;
            bi = i;
        }
    if (bi >= 0) {
        void *p = s->pinned_free[bi].first;
        s->pinned_free.erase(s->pinned_free.begin() + bi);
        return p;
    }
    void *p = nullptr;
    if (cudaMallocHost(&p, n) != cudaSuccess) return nullptr;
    return p;
}

void pinned_put(gfc_server *s, void *p, size_t n)
{
    if (p) s->pinned_free.push_back({p, n});
}

double work_per_point(const Request &r, int arith)
{
    double nodes = r.params.n_radial;
    if (r.prop.kind != GFC_PROP_SCALAR) nodes *= 1.75;
    double terms = r.prop.kind == GFC_PROP_DRESSED ? 2.0 : 1.0;
    // the closed-form angular integral costs about as much as four pairs
    double w = nodes * std::max(npair_of(&r.params), 4) * terms;
    return arith == ARITH_F32 ? w : (arith == ARITH_DF ? w * kDfWeight : w * kFp64Weight);
}

// Estimated work of a whole request (binary32-pair units): every point in its
// arithmetic; for mixed precision the binary32 bulk and the expected fallback.
double request_work(const Request &r)
{
    if (r.params.precision != GFC_MIXED) {
        const int ar = r.params.precision == GFC_F32X2 ? ARITH_DF : ARITH_F64;
        return r.npts * work_per_point(r, ar);
    }
    const int fb = r.params.mixed_fallback == GFC_F32X2 ? ARITH_DF : ARITH_F64;
    return r.npts * (work_per_point(r, ARITH_F32) + kMixedRouted * work_per_point(r, fb));
}

// Scheduling key: the least first (shortest remaining work, aged by waiting).
double sched_key(const Request &r, clk::time_point now)
{
    const double wait = std::chrono::duration<double>(now - r.t_submit).count();
    return r.work_left - kAgeRate * wait;
}

void release_request(gfc_server *s, Request *r)
{
    if (r->G_dev && !r->G_on_device) cudaFreeAsync(r->G_dev, s->admit_stream);
    r->G_dev = nullptr;
    if (r->list_dev) cudaFreeAsync(r->list_dev, s->admit_stream);
    r->list_dev = nullptr;
    if (r->count_done) cudaEventDestroy(r->count_done);
    r->count_done = nullptr;
    if (r->pinned) pinned_put(s, r->pinned, r->pinned_size);
    r->pinned = nullptr;
    if (r->copy_done) cudaEventDestroy(r->copy_done);
    r->copy_done = nullptr;
    if (r->slot >= 0) s->free_slots.push_back(r->slot);
    r->slot = -1;
    s->bytes_in_use -= r->bytes;
    s->active.erase(std::remove(s->active.begin(), s->active.end(), r), s->active.end());
}

// Marks a request whose work or copies hit a CUDA error: no further work is
// scheduled for it, and once nothing of it is in flight it finishes with
// GFC_ECUDA (its output is never reported as a result).
void mark_failed(Request *r, const std::string &msg)
{
    if (!r->failed) r->fail_msg = msg;
    r->failed = true;
}

std::string cuda_msg(const char *what, cudaError_t e)
{
    return std::string(what) + ": " + cudaGetErrorName(e);
}

void finish(gfc_server *s, Request *r, int status)
{
    r->status = status;
    r->state = R_DONE;
    r->t_done = clk::now();
    if (status == GFC_OK) {
        s->n_completed++;
        s->points_done += r->npts;
        s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
        if (!s->any_done) s->t_first = r->t_submit;
        s->any_done = true;
        s->t_last = r->t_done;
    } else if (status == GFC_ECANCELED) {
        s->n_canceled++;
    }
    s->cv_done.notify_all();
}

// Admission: slot, output buffer, descriptor upload and G0(mu2).
int admit(gfc_server *s, Request *r)
{
    int rc = get_tables_c(s->device, r->params.n_radial, r->params.n_angular, r->params.dim,
                          r->params.radial_scale, r->params.angular_rule, &r->T, nullptr);
    if (rc) return rc;
    PropConst pc;
    if ((rc = make_prop_c(&r->prop, &r->params, pc))) return rc;
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    cudaError_t e = cudaSuccess;
    if (r->G_on_device) {
        r->G_dev = r->G_host;   // the caller's device array receives the grid directly
    } else {
        e = dev_malloc_async((void **)&r->G_dev, 16 * r->npts, s->admit_stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(request output)");
    }
    const bool mixed = r->params.precision == GFC_MIXED;
    if (mixed) {
        e = dev_malloc_async((void **)&r->list_dev, sizeof(int64_t) * r->npts, s->admit_stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(request list)");
        e = cudaMemsetAsync(s->slot_counts_dev + r->slot, 0, sizeof(unsigned long long),
                            s->admit_stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(list length)");
        if (cudaEventCreateWithFlags(&r->count_done, cudaEventDisableTiming) != cudaSuccess)
            return fail(GFC_ECUDA, "cudaEventCreate");
    }
    KParams &kp = r->kp;
    fill_kparams_c(kp, &r->params, *r->T, pc);
    kp.use_grid = 1;
    kp.npts = r->npts;
    kp.re0 = r->grid.re0;
    kp.dre = (r->grid.re1 - r->grid.re0) / r->grid.m;
    kp.im0 = r->grid.im0;
    kp.dim_im = (r->grid.im1 - r->grid.im0) / r->grid.n;
    kp.gm = r->grid.m;
    kp.gn = r->grid.n;
    kp.G = r->G_dev;
    kp.g0mu = s->g0mu_dev + 2 * r->slot;
    kp.counter = nullptr;
    kp.node_count = nullptr;
    kp.list = r->list_dev;
    kp.list_count = mixed ? s->slot_counts_dev + r->slot : nullptr;
    kp.cond_out = nullptr;
    s->slots_host[r->slot] = kp;
    e = cudaMemcpyAsync(s->slots_dev + r->slot, s->slots_host + r->slot, sizeof(KParams),
                        cudaMemcpyHostToDevice, s->admit_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync(slot)");
    DevTables tb = dev_tables_c(*r->T);
    int nw = (r->params.n_radial + 31) / 32;
    if (nw > kG0Warps) nw = kG0Warps;
    e = launch_g0mu(kp, tb, r->params.mu2, s->partials_dev, nw, s->ticket_dev,
                    s->g0mu_dev + 2 * r->slot, s->dummy_counters, s->admit_stream);
    if (e != cudaSuccess) return cuda_fail(e, "g0mu launch");
    e = cudaEventRecord(s->admit_event, s->admit_stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(admission)");
    if (!mixed) {
        int ar = r->params.precision == GFC_F32X2 ? ARITH_DF : ARITH_F64;
        r->phases = {Phase{MODE_ALL, ar, 0, r->npts, 0}};
    } else {
        int ar = r->params.mixed_fallback == GFC_F32X2 ? ARITH_DF : ARITH_F64;
        r->phases = {Phase{MODE_BULK32, ARITH_F32, 0, r->npts, 0}, Phase{MODE_LIST64, ar, 0, -1, 0}};
    }
    r->state = R_ACTIVE;
    r->admitted = true;
    r->t_admit = clk::now();
    s->active.push_back(r);
    return GFC_OK;
}

bool request_complete(const Request *r)
{
    for (const Phase &ph : r->phases)
        if (ph.end < 0 || ph.next < ph.end || ph.items_out > 0) return false;
    return true;
}

// Batched launches, one per kernel variant with pending points, the variant
// whose most urgent request (least sched_key) ranks first going first, while
// fewer than kMaxInflight launches are on the device. Within a launch the
// variant's requests are served least key first (shortest remaining work,
// aged), each up to the launch's work budget; a launch whose first request
// is urgent (key below two launches of work) goes to a high-priority stream,
// so that its blocks start ahead of those of launches for longer requests.
void issue_launches(gfc_server *s)
{
    const clk::time_point now = clk::now();
    std::map<GroupKey, std::vector<std::pair<Request *, int>>> groups;
    for (Request *r : s->active) {
        if (r->canceled || r->failed) continue;
        for (int p = 0; p < (int)r->phases.size(); ++p) {
            const Phase &ph = r->phases[p];
            if (ph.end < 0 || ph.next >= ph.end) continue;
            GroupKey k{ph.arith, npair_of(&r->params), r->params.dim,
                       r->prop.kind == GFC_PROP_DRESSED ? 1 : 0, ph.mode, r->params.angular_rule,
                       r->params.radial_rule};
            groups[k].push_back({r, p});
        }
    }
    // the groups in the order of their most urgent request, each group's
    // requests least key first
    std::vector<std::pair<double, GroupKey>> order;
    for (auto &kv : groups) {
        auto &members = kv.second;
        std::stable_sort(members.begin(), members.end(), [now](const auto &a, const auto &b) {
            return sched_key(*a.first, now) < sched_key(*b.first, now);
        });
        order.push_back({sched_key(*members.front().first, now), kv.first});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const auto &a, const auto &b) { return a.first < b.first; });
    int inflight = 0;
    for (int i = 0; i < kRing; ++i) inflight += s->ring[i].busy ? 1 : 0;
    for (auto &og : order) {
        if (inflight >= kMaxInflight) return;
        int li = -1;
        for (int i = 0; i < kRing; ++i)
            if (!s->ring[i].busy) {
                li = i;
                break;
            }
        if (li < 0) return;
        LaunchRec &L = s->ring[li];
        const GroupKey &key = og.second;
        const int arith = std::get<0>(key);
        const int mode = std::get<4>(key);
        auto &members = groups[key];
        const bool urgent = og.first < 2.0 * kLaunchWork;
        // least key first, each request up to what the budget has left
        double budget = kLaunchWork;
        int nitems = 0;
        int64_t total = 0;
        L.reqs.clear();
        std::map<std::pair<Request *, int>, int64_t> count;
        for (auto &m : members) {
            if (budget <= 0 || nitems >= kMaxItems) break;
            Request *r = m.first;
            Phase &ph = r->phases[m.second];
            const double wpp = work_per_point(*r, arith);
            // items of at least 256 points (or what is left), at most the budget
            int64_t n = (int64_t)std::max(256.0, budget / wpp);
            n = std::min(n, ph.end - ph.next);
            if (n <= 0) continue;
            L.items_host[nitems] = BatchItem{r->slot, 0, ph.next, ph.next + n};
            L.offs_host[nitems] = total;
            total += n;
            ph.next += n;
            budget -= n * wpp;
            r->work_left = std::max(0.0, r->work_left - n * wpp);
            count[{r, m.second}] += 1;
            ++nitems;
        }
        if (nitems == 0) continue;
        ++inflight;
        for (auto &c : count) {
            c.first.first->phases[c.first.second].items_out += c.second;
            c.first.first->launches++;
            L.reqs.push_back(std::make_tuple(c.first.first, c.first.second, c.second));
        }
        // high-priority streams 0 and 1, low-priority 2 and 3, alternating
        const int si = (urgent ? 0 : 2) + (s->next_stream++ & 1);
        cudaStream_t st = s->streams[si];
        L.failed = false;
        L.fail_msg.clear();
        auto chk = [&L](cudaError_t e, const char *what) {
            if (e != cudaSuccess && !L.failed) {
                L.failed = true;
                L.fail_msg = cuda_msg(what, e);
            }
        };
        chk(cudaStreamWaitEvent(st, s->admit_event, 0), "cudaStreamWaitEvent");
        chk(cudaMemcpyAsync(L.items_dev, L.items_host, sizeof(BatchItem) * nitems,
                            cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(items)");
        chk(cudaMemcpyAsync(L.offs_dev, L.offs_host, sizeof(int64_t) * nitems,
                            cudaMemcpyHostToDevice, st), "cudaMemcpyAsync(offsets)");
        chk(cudaMemsetAsync(L.counter_dev, 0, sizeof(unsigned long long), st),
            "cudaMemsetAsync(counter)");
        BatchLaunch bl;
        bl.slots = s->slots_dev;
        bl.items = L.items_dev;
        bl.offs = L.offs_dev;
        bl.nitems = nitems;
        bl.total = total;
        bl.counter = L.counter_dev;
        bl.mode = mode;
        bl.npair = std::get<1>(key);
        Request *r0 = members.front().first;
        bl.rules_total = r0->kp.rules_total;
        bl.radial_rule = std::get<6>(key);
        bl.ang_exact = std::get<5>(key) == GFC_ANG_EXACT;
        nvtxRangePushA("gfc_server_launch");
        // nothing is launched after a failed copy: the launch would read stale items
        if (!L.failed) chk(launch_batch(bl, dev_tables_c(*r0->T), arith, std::get<3>(key) != 0, st),
                           "batched launch");
        nvtxRangePop();
        if (L.failed) s->error = GFC_ECUDA;
        chk(cudaEventRecord(L.done, st), "cudaEventRecord(launch)");
        L.busy = true;
        s->launches++;
    }
}

// Retire finished launches and copies; returns true if anything changed.
bool progress(gfc_server *s)
{
    bool changed = false;
    for (int i = 0; i < kRing; ++i) {
        LaunchRec &L = s->ring[i];
        if (!L.busy) continue;
        cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) continue;
        // an error of the launch itself (or of the calls that issued it)
        // fails every request the launch carried
        const bool bad = L.failed || q != cudaSuccess;
        const std::string msg = L.failed ? L.fail_msg : cuda_msg("batched launch", q);
        L.busy = false;
        L.failed = false;
        changed = true;
        for (auto &rc : L.reqs) {
            Request *r = std::get<0>(rc);
            r->phases[std::get<1>(rc)].items_out -= std::get<2>(rc);
            if (bad) mark_failed(r, msg);
        }
        L.reqs.clear();
    }
    std::vector<Request *> act = s->active;
    for (Request *r : act) {
        if (r->state != R_ACTIVE) goto copying;
        if (r->phases.size() == 2) {
            // mixed: once the binary32 phase is done, read the list length
            Phase &p0 = r->phases[0], &p1 = r->phases[1];
            if (r->count_pending) {
                const cudaError_t q = cudaEventQuery(r->count_done);
                if (q == cudaSuccess) {
                    p1.end = (int64_t)s->slot_counts_host[r->slot];
                    r->routed = p1.end;
                    r->work_left = p1.end * work_per_point(*r, p1.arith);
                    r->count_pending = false;
                    changed = true;
                } else if (q != cudaErrorNotReady) {
                    mark_failed(r, cuda_msg("routed-point count", q));
                    r->count_pending = false;
                    changed = true;
                }
            } else if (!r->canceled && !r->failed && p1.end < 0 && p0.next >= p0.end &&
                       p0.items_out == 0) {
                cudaError_t e = cudaMemcpyAsync(s->slot_counts_host + r->slot,
                                                s->slot_counts_dev + r->slot,
                                                sizeof(unsigned long long),
                                                cudaMemcpyDeviceToHost, s->copy_stream);
                if (e == cudaSuccess) e = cudaEventRecord(r->count_done, s->copy_stream);
                if (e == cudaSuccess) r->count_pending = true;
                else mark_failed(r, cuda_msg("routed-point count copy", e));
                changed = true;
            }
        }
        {
            bool idle = true;
            for (const Phase &ph : r->phases) idle = idle && ph.items_out == 0;
            if ((r->canceled || r->failed) && idle && !r->count_pending) {
                release_request(s, r);
                if (r->canceled) {
                    finish(s, r, GFC_ECANCELED);
                } else {
                    finish(s, r, GFC_ECUDA);
                }
                changed = true;
                continue;
            }
        }
    copying:
        if (r->state == R_ACTIVE && !r->canceled && !r->failed && request_complete(r) &&
            r->G_on_device) {
            // the kernels wrote the caller's device array; every launch of the
            // request has retired, so the result is complete
            release_request(s, r);
            finish(s, r, GFC_OK);
            changed = true;
        } else if (r->state == R_ACTIVE && !r->canceled && !r->failed && request_complete(r)) {
            r->pinned_size = 16 * r->npts;
            r->pinned = pinned_get(s, r->pinned_size);
            if (!r->pinned || cudaEventCreateWithFlags(&r->copy_done, cudaEventDisableTiming)) {
                release_request(s, r);
                finish(s, r, GFC_ENOMEM);
                continue;
            }
            cudaError_t e = cudaMemcpyAsync(r->pinned, r->G_dev, r->pinned_size,
                                            cudaMemcpyDeviceToHost, s->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(r->copy_done, s->copy_stream);
            if (e != cudaSuccess) {
                release_request(s, r);
                r->fail_msg = cuda_msg("result copy", e);
                finish(s, r, GFC_ECUDA);
                changed = true;
                continue;
            }
            r->state = R_COPYING;
            changed = true;
        } else if (r->state == R_COPYING) {
            const cudaError_t q = cudaEventQuery(r->copy_done);
            if (q == cudaErrorNotReady) continue;
            const bool ok = q == cudaSuccess;
            if (ok && !r->canceled) std::memcpy(r->G_host, r->pinned, r->pinned_size);
            release_request(s, r);
            if (!ok) r->fail_msg = cuda_msg("result copy", q);
            finish(s, r, r->canceled ? GFC_ECANCELED : (ok ? GFC_OK : GFC_ECUDA));
            changed = true;
        }
    }
    return changed;
}

void scheduler(gfc_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        // admission: the queued request with the least key (shortest work,
        // aged by waiting) that fits the budget, while slots are free
        while (!s->queue.empty() && !s->free_slots.empty()) {
            const clk::time_point now = clk::now();
            auto best = s->queue.end();
            double bk = 0.0;
            for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
                if ((*it)->canceled || s->bytes_in_use + (*it)->bytes > s->budget) continue;
                const double k = sched_key(**it, now);
                if (best == s->queue.end() || k < bk) {
                    best = it;
                    bk = k;
                }
            }
            if (best == s->queue.end()) break;
            Request *r = *best;
            s->queue.erase(best);
            s->bytes_in_use += r->bytes;
            int rc = admit(s, r);
            if (rc != GFC_OK) {
                release_request(s, r);
                finish(s, r, rc);
            }
        }
        issue_launches(s);
        bool changed = progress(s);
        bool busy = !s->active.empty();
        for (int i = 0; i < kRing && !busy; ++i) busy = s->ring[i].busy;
        if (s->stopping && s->queue.empty() && !busy) break;
        if (!busy && s->queue.empty()) {
            s->cv_work.wait_for(lk, std::chrono::milliseconds(20));
        } else if (!changed) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(100));
            lk.lock();
        }
    }
}

}  // namespace
}  // namespace gfc

using namespace gfc;

extern "C" {

int gfc_server_create(int device, size_t hbm_budget_bytes, int max_slots, gfc_server **out)
{
    if (!out) return fail(GFC_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 4096) return fail(GFC_EINVAL, "max_slots must be in [1, 4096]");
    if (hbm_budget_bytes < (1u << 20)) return fail(GFC_EINVAL, "budget below 1 MiB");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(GFC_EINVAL, "no such device");
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    auto s = std::make_unique<gfc_server>();
    s->device = device;
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    for (int i = max_slots - 1; i >= 0; --i) s->free_slots.push_back(i);
    bool ok = cudaStreamCreateWithFlags(&s->admit_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&s->admit_event, cudaEventDisableTiming) == cudaSuccess;
    // launch streams: two at the device's greatest priority, two at its least
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    for (int i = 0; i < kStreams && ok; ++i)
        ok = cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking,
                                          i < 2 ? prio_hi : prio_lo) == cudaSuccess;
    ok = ok && cudaMalloc((void **)&s->slots_dev, sizeof(KParams) * max_slots) == cudaSuccess &&
         cudaMallocHost((void **)&s->slots_host, sizeof(KParams) * max_slots) == cudaSuccess &&
         cudaMalloc((void **)&s->g0mu_dev, sizeof(double) * 2 * max_slots) == cudaSuccess &&
         cudaMalloc((void **)&s->slot_counts_dev, sizeof(unsigned long long) * max_slots) == cudaSuccess &&
         cudaMallocHost((void **)&s->slot_counts_host, sizeof(unsigned long long) * max_slots) == cudaSuccess &&
         cudaMalloc((void **)&s->partials_dev, sizeof(double) * 2 * kG0Warps) == cudaSuccess &&
         cudaMalloc((void **)&s->ticket_dev, sizeof(unsigned)) == cudaSuccess &&
         cudaMemset(s->ticket_dev, 0, sizeof(unsigned)) == cudaSuccess &&
         cudaMalloc((void **)&s->dummy_counters, sizeof(unsigned long long) * kCounters) == cudaSuccess;
    for (int i = 0; i < kRing && ok; ++i) {
        LaunchRec &L = s->ring[i];
        ok = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) == cudaSuccess &&
             cudaMalloc((void **)&L.items_dev, sizeof(BatchItem) * kMaxItems) == cudaSuccess &&
             cudaMalloc((void **)&L.offs_dev, sizeof(int64_t) * kMaxItems) == cudaSuccess &&
             cudaMalloc((void **)&L.counter_dev, sizeof(unsigned long long)) == cudaSuccess &&
             cudaMallocHost((void **)&L.items_host, sizeof(BatchItem) * kMaxItems) == cudaSuccess &&
             cudaMallocHost((void **)&L.offs_host, sizeof(int64_t) * kMaxItems) == cudaSuccess;
    }
    // the budget bounds what admitted requests hold (outputs and lists); the
    // server's own fixed tables (slots, launch rings) are outside it
    s->bytes_in_use = 0;
    if (!ok) {
        gfc_server *raw = s.release();
        gfc_server_destroy(raw);
        return fail(GFC_ENOMEM, "server allocation failed");
    }
    gfc_server *raw = s.release();
    raw->th = std::thread(scheduler, raw);
    *out = raw;
    return GFC_OK;
}

int gfc_server_submit(gfc_server *s, const gfc_propagator *prop, const gfc_params *params,
                      const gfc_grid *grid, double *G_host, uint64_t *ticket)
{
    if (!s || !ticket || !G_host) return fail(GFC_EINVAL, "NULL argument");
    int rc = check_params_c(params);
    if (rc) return rc;
    if ((rc = check_grid_c(grid))) return rc;
    PropConst pc;
    if ((rc = make_prop_c(prop, params, pc))) return rc;
    auto r = std::make_unique<Request>();
    r->prop = *prop;
    r->params = *params;
    r->grid = *grid;
    r->G_host = G_host;
    r->npts = (int64_t)grid->m * grid->n;
    {
        // device memory of the server's device is written in place; anything
        // else is host memory that receives a copy
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, G_host) == cudaSuccess &&
            (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
            if (a.type == cudaMemoryTypeDevice && a.device != s->device)
                return fail(GFC_EINVAL, "G is device memory of another device");
            r->G_on_device = a.type == cudaMemoryTypeDevice;
        }
        cudaGetLastError();
    }
    // the server holds the output grid (host outputs) and the routed list (mixed)
    r->bytes = ((r->G_on_device ? 0 : 16) + (params->precision == GFC_MIXED ? 8 : 0)) *
               (size_t)r->npts;
    r->t_submit = clk::now();
    r->work_left = request_work(*r);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return fail(GFC_EBUSY, "server is shutting down");
    if (r->bytes > s->budget) {
        s->n_rejected++;
        return fail(GFC_EBUDGET, "request exceeds the memory budget");
    }
    r->ticket = s->next_ticket++;
    *ticket = r->ticket;
    s->queue.push_back(r.get());
    s->reqs[r->ticket] = std::move(r);
    s->n_submitted++;
    s->cv_work.notify_all();
    return GFC_OK;
}

int gfc_server_poll(gfc_server *s, uint64_t ticket, int *done, int *status)
{
    if (!s || !done || !status) return fail(GFC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GFC_ENOTFOUND, "unknown ticket");
    *done = it->second->state == R_DONE;
    *status = *done ? it->second->status : GFC_OK;
    return GFC_OK;
}

int gfc_server_wait(gfc_server *s, uint64_t ticket, int timeout_ms)
{
    if (!s) return fail(GFC_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GFC_ENOTFOUND, "unknown ticket");
    Request *r = it->second.get();
    auto pred = [r] { return r->state == R_DONE; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        return fail(GFC_ETIMEOUT, "request still running");
    }
    if (r->status == GFC_ECUDA && !r->fail_msg.empty()) fail(GFC_ECUDA, r->fail_msg.c_str());
    return r->status;
}

int gfc_server_request_info(gfc_server *s, uint64_t ticket, gfc_request_info *out)
{
    if (!s || !out) return fail(GFC_EINVAL, "NULL server or output");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GFC_ENOTFOUND, "unknown ticket");
    const Request *r = it->second.get();
    auto ms = [](clk::time_point a, clk::time_point b) {
        return std::chrono::duration<double, std::milli>(b - a).count();
    };
    out->status = r->state == R_DONE ? r->status : GFC_ETIMEOUT;
    out->state = r->state == R_QUEUED ? 0 : (r->state == R_DONE ? 2 : 1);
    out->points = r->npts;
    out->points_routed = r->routed;
    out->queue_ms = r->admitted ? ms(r->t_submit, r->t_admit) : -1.0;
    out->total_ms = r->state == R_DONE ? ms(r->t_submit, r->t_done) : -1.0;
    out->launches = r->launches;
    out->bytes = r->bytes;
    return GFC_OK;
}

int gfc_server_cancel(gfc_server *s, uint64_t ticket)
{
    if (!s) return fail(GFC_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(GFC_ENOTFOUND, "unknown ticket");
    Request *r = it->second.get();
    if (r->state == R_DONE) return fail(GFC_EINVAL, "request already finished");
    r->canceled = true;
    if (r->state == R_QUEUED) {
        s->queue.erase(std::remove(s->queue.begin(), s->queue.end(), r), s->queue.end());
        finish(s, r, GFC_ECANCELED);
    }
    // an active request stops being scheduled and is released once its
    // launched items finish; a copying request's host buffer is not written
    s->cv_work.notify_all();
    return GFC_OK;
}

int gfc_server_stats(gfc_server *s, gfc_stats *out)
{
    if (!s || !out) return fail(GFC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = s->n_submitted;
    out->completed = s->n_completed;
    out->rejected = s->n_rejected;
    out->canceled = s->n_canceled;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&v](double q) {
            size_t k = (size_t)std::ceil(q * v.size()) - 1;
            return v[std::min(k, v.size() - 1)];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    if (s->any_done) {
        double sec = std::chrono::duration<double>(s->t_last - s->t_first).count();
        out->points_per_s = sec > 0 ? s->points_done / sec : 0.0;
    }
    out->points_done = s->points_done;
    out->bytes_in_use = s->bytes_in_use;
    out->bytes_budget = s->budget;
    out->launches = s->launches;
    out->queued = (int)s->queue.size();
    out->active = (int)s->active.size();
    return GFC_OK;
}

int gfc_server_load(gfc_server *s, double *work)
{
    if (!s || !work) return fail(GFC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    double w = 0.0;
    for (const Request *r : s->queue) w += r->work_left;
    for (const Request *r : s->active) w += r->work_left;
    *work = w;
    return GFC_OK;
}

int gfc_server_destroy(gfc_server *s)
{
    if (!s) return fail(GFC_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        for (Request *r : s->queue) {
            r->canceled = true;
            finish(s, r, GFC_ECANCELED);
        }
        s->queue.clear();
        s->cv_work.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    cudaSetDevice(s->device);
    if (s->admit_stream) cudaStreamSynchronize(s->admit_stream);
    for (int i = 0; i < kRing; ++i) {
        LaunchRec &L = s->ring[i];
        if (L.done) cudaEventDestroy(L.done);
        cudaFree(L.items_dev);
        cudaFree(L.offs_dev);
        cudaFree(L.counter_dev);
        cudaFreeHost(L.items_host);
        cudaFreeHost(L.offs_host);
    }
    for (auto &p : s->pinned_free) cudaFreeHost(p.first);
    cudaFree(s->slots_dev);
    cudaFreeHost(s->slots_host);
    cudaFree(s->g0mu_dev);
    cudaFree(s->slot_counts_dev);
    cudaFreeHost(s->slot_counts_host);
    cudaFree(s->partials_dev);
    cudaFree(s->ticket_dev);
    cudaFree(s->dummy_counters);
    for (int i = 0; i < kStreams; ++i)
        if (s->streams[i]) cudaStreamDestroy(s->streams[i]);
    if (s->admit_stream) cudaStreamDestroy(s->admit_stream);
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    if (s->admit_event) cudaEventDestroy(s->admit_event);
    delete s;
    return GFC_OK;
}

}  // extern "C"
