// Requests over several devices: one continuous-batching server per device,
// each request handed whole to the server with the least estimated work
// outstanding (queued and admitted work not yet launched). Every point is
// independent, so a request needs nothing from the other devices; tickets
// carry the index of the server that holds the request.
#include <cstdint>
#include <memory>
#include <mutex>
#include <vector>

#include "gfc.h"
#include "gfc_internal.h"

struct gfc_router {
    std::vector<gfc_server *> servers;
    std::mutex mu;
};

namespace {

constexpr int kMaxServers = 256;   // a ticket keeps the server index in its low 8 bits

int split(gfc_router *r, uint64_t ticket, gfc_server **s, uint64_t *t)
{
    const int i = (int)(ticket & 0xffu);
    if (!r || i >= (int)r->servers.size()) return gfc::fail(GFC_ENOTFOUND, "unknown ticket");
    *s = r->servers[i];
    *t = ticket >> 8;
    return GFC_OK;
}

}  // namespace

extern "C" {

int gfc_router_create(const int *devices, int ndevices, size_t hbm_budget_bytes, int max_slots,
                      gfc_router **out)
{
    if (!out || !devices) return gfc::fail(GFC_EINVAL, "NULL argument");
    *out = nullptr;
    if (ndevices < 1 || ndevices > kMaxServers)
        return gfc::fail(GFC_EINVAL, "ndevices must be in [1, 256]");
    auto r = std::make_unique<gfc_router>();
    for (int i = 0; i < ndevices; ++i) {
        gfc_server *s = nullptr;
        const int rc = gfc_server_create(devices[i], hbm_budget_bytes, max_slots, &s);
        if (rc) {
            for (gfc_server *t : r->servers) gfc_server_destroy(t);
            return rc;
        }
        r->servers.push_back(s);
    }
    *out = r.release();
    return GFC_OK;
}

int gfc_router_submit(gfc_router *r, const gfc_propagator *prop, const gfc_params *params,
                      const gfc_grid *grid, double *G_host, uint64_t *ticket)
{
    if (!r || !ticket) return gfc::fail(GFC_EINVAL, "NULL argument");
    // one submission at a time, so that two requests do not both pick the
    // server that was least loaded before either arrived
    std::lock_guard<std::mutex> lk(r->mu);
    int best = 0;
    double best_w = 0.0;
    for (int i = 0; i < (int)r->servers.size(); ++i) {
        double w = 0.0;
        const int rc = gfc_server_load(r->servers[i], &w);
        if (rc) return rc;
        if (i == 0 || w < best_w) {
            best = i;
            best_w = w;
        }
    }
    uint64_t t = 0;
    const int rc = gfc_server_submit(r->servers[best], prop, params, grid, G_host, &t);
    if (rc) return rc;
    *ticket = (t << 8) | (uint64_t)best;
    return GFC_OK;
}

int gfc_router_poll(gfc_router *r, uint64_t ticket, int *done, int *status)
{
    gfc_server *s;
    uint64_t t;
    const int rc = split(r, ticket, &s, &t);
    return rc ? rc : gfc_server_poll(s, t, done, status);
}

int gfc_router_wait(gfc_router *r, uint64_t ticket, int timeout_ms)
{
    gfc_server *s;
    uint64_t t;
    const int rc = split(r, ticket, &s, &t);
    return rc ? rc : gfc_server_wait(s, t, timeout_ms);
}

int gfc_router_cancel(gfc_router *r, uint64_t ticket)
{
    gfc_server *s;
    uint64_t t;
    const int rc = split(r, ticket, &s, &t);
    return rc ? rc : gfc_server_cancel(s, t);
}

int gfc_router_server(gfc_router *r, int index, gfc_server **out)
{
    if (!r || !out) return gfc::fail(GFC_EINVAL, "NULL argument");
    if (index < 0 || index >= (int)r->servers.size()) return gfc::fail(GFC_EINVAL, "no such server");
    *out = r->servers[index];
    return GFC_OK;
}

int gfc_router_server_of(gfc_router *r, uint64_t ticket, int *index, uint64_t *server_ticket)
{
    if (!index || !server_ticket) return gfc::fail(GFC_EINVAL, "NULL argument");
    gfc_server *s;
    const int rc = split(r, ticket, &s, server_ticket);
    if (rc) return rc;
    *index = (int)(ticket & 0xffu);
    return GFC_OK;
}

int gfc_router_destroy(gfc_router *r)
{
    if (!r) return gfc::fail(GFC_EINVAL, "NULL router");
    for (gfc_server *s : r->servers) gfc_server_destroy(s);
    delete r;
    return GFC_OK;
}

}  // extern "C"
