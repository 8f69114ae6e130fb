// Served form: continuous batching of expansion requests (host runtime).
//
// One context is shared by every server thread: the context's caches, pools
// and launch decisions are guarded, each request's handles are used by one
// thread at a time (its prep thread, then the launcher), and device memory
// shared between requests (cached geometries and enumerations) is released
// only after every stream that used it.
//
// Requests arrive as single networks of any size, bond dimension and order.
// They are admitted in arrival order while the estimated device bytes and the
// number of admitted, unfinished requests stay within the server's budget.
// Prep threads (each with its own stream) build the partition (BP, gauge) and
// the enumeration of an admitted request -- the latter from the context's
// geometry cache when another request of the same geometry came before --
// while a launcher thread takes every request that is ready and runs them in
// one fused persistent launch (contractions + term sums, Sec. II.D: all terms
// in parallel).  Requests that arrive meanwhile are admitted and prepared
// concurrently and join the following launch.  A request's arithmetic never
// depends on its neighbours in a launch, so its result is the same alone and
// in a mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "pne_internal.h"

namespace {

struct Request {
    uint64_t id = 0;
    int n_sites = 0, n_bonds = 0, K = 0;
    std::vector<int32_t> bond_site, bond_dim, site_ptr, site_bonds;
    std::vector<double> data;
    std::vector<int64_t> data_off;
    uint64_t est_bytes = 0;
    pne_partition *part = nullptr;
    pne_terms *terms = nullptr;
    pne_result result{};
    pne_status status = PNE_OK;
    pne_request_info info{};
    bool done = false;
};

uint64_t fnv(uint64_t h, const void *p, size_t n)
{
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

}  // namespace

struct pne_server {
    pne_ctx *ctx = nullptr;
    pne_server_opts opts{};
    std::mutex mu;
    std::condition_variable cv_admit, cv_ready, cv_done;
    std::deque<Request *> arrivals, ready;
    std::unordered_map<uint64_t, Request *> all;
    uint64_t next_id = 1, inflight_bytes = 0, peak_bytes = 0;
    int inflight = 0, outstanding = 0;
    bool stop = false;
    std::vector<std::thread> prep;
    std::thread launcher;
    std::vector<cudaStream_t> streams;
    cudaStream_t launch_stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    std::string first_error;      // message of the first failed request

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Device bytes a request will hold until it completes: tensors (raw, blocked,
// converted), messages and gauges, plus clusters, terms and cluster values --
// from the geometry cache when present, else a growth estimate.
uint64_t estimate_bytes(pne_server *s, const Request &r)
{
    const uint64_t entries = (uint64_t)r.data.size();
    const uint64_t legs = (uint64_t)r.site_bonds.size();
    uint64_t b = entries * (8 + 8 + 4) + legs * 2 * 8 * 8 + (uint64_t)r.n_bonds * 2 * 64 * 8 + (uint64_t)r.n_sites * 96;
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &r.n_sites, sizeof r.n_sites);
    h = fnv(h, r.bond_site.data(), r.bond_site.size() * 4);
    h = fnv(h, r.bond_dim.data(), r.bond_dim.size() * 4);
    const std::string key = std::to_string(h) + ":" + std::to_string(r.n_sites) + ":" + std::to_string(r.n_bonds) + ":" +
                            std::to_string(r.K) + ":" + std::to_string((int)PNE_MODE_LOOP);
    uint64_t n_cl = 0, n_t = 0;
    {
        std::lock_guard<std::mutex> lk(s->ctx->cache_mu);
        auto it = s->ctx->enum_cache.find(key);
        if (it != s->ctx->enum_cache.end()) { n_cl = it->second->n_clusters; n_t = it->second->n_terms; }
    }
    if (n_cl == 0) {                      // not cached yet: a generous per-bond growth
        n_cl = (uint64_t)r.n_bonds * (1ull << std::min(r.K, 16)) / 4 + 1;
        n_t = n_cl * 8;
    }
    b += n_cl * (uint64_t)(4 * r.K + 4 * (r.K + 1) + 4 + 8 + 4 + 16) + n_t * 8;
    return b;
}

bool fits(pne_server *s, const Request &r)
{
    if (s->inflight >= s->opts.max_inflight) return false;
    if (s->inflight == 0) return true;                 // never starve an oversized request
    return s->inflight_bytes + r.est_bytes <= s->opts.device_budget_bytes;
}

void finish_locked(pne_server *s, Request *r, pne_status st)
{
    if (st != PNE_OK && s->first_error.empty()) {
        // the failing call ran in this thread: its message is this thread's
        s->first_error = std::string("request ") + std::to_string(r->id) + ": " + pne_last_error(s->ctx);
        if (s->first_error.empty()) s->first_error = "status " + std::to_string((int)st);
    }
    r->status = st;
    r->done = true;
    r->info.t_done = s->now();
    s->inflight -= 1;
    s->inflight_bytes -= r->est_bytes;
    s->outstanding -= 1;
}

void release(Request *r)
{
    if (r->terms) { pne_terms_destroy(r->terms); r->terms = nullptr; }
    if (r->part) { pne_partition_destroy(r->part); r->part = nullptr; }
}

void prep_loop(pne_server *s, int w)
{
    cudaSetDevice(s->ctx->device);
    cudaStream_t st = s->streams[w];
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_admit.wait(lk, [&] { return s->stop || (!s->arrivals.empty() && fits(s, *s->arrivals.front())); });
            if (s->stop) return;
            r = s->arrivals.front();
            s->arrivals.pop_front();
            s->inflight += 1;
            s->inflight_bytes += r->est_bytes;
            s->peak_bytes = std::max(s->peak_bytes, s->inflight_bytes);
            r->info.t_admit = s->now();
        }
        pne_network net;
        net.n_sites = r->n_sites; net.n_bonds = r->n_bonds;
        net.bond_site = r->bond_site.data(); net.bond_dim = r->bond_dim.data();
        net.site_ptr = r->site_ptr.data(); net.site_bonds = r->site_bonds.data();
        net.data = r->data.data(); net.data_off = r->data_off.data();
        net.data_on_device = 0; net.n_batch = 1;
        // float-float sweeps: one thread-block cluster per network, so the
        // partitions of several requests run side by side on the FP32 pipes
        pne_partition_opts po{1e-13, 10000, 0.0, 1, 0};
        pne_status rc = pne_build_partition(s->ctx, &net, &po, st, &r->part);
        if (rc == PNE_OK) {
            pne_enum_opts eo{r->K, PNE_MODE_LOOP, 1};
            rc = pne_enumerate_terms(s->ctx, r->part, &eo, st, &r->terms, nullptr, nullptr);
        }
        // the host copy of the tensors is no longer needed
        std::vector<double>().swap(r->data);
        std::unique_lock<std::mutex> lk(s->mu);
        r->info.t_ready = s->now();
        if (rc != PNE_OK) {
            release(r);
            finish_locked(s, r, rc);
            s->cv_admit.notify_all();
            s->cv_done.notify_all();
        } else {
            s->ready.push_back(r);
            s->cv_ready.notify_one();
        }
    }
}

void launch_loop(pne_server *s)
{
    cudaSetDevice(s->ctx->device);
    for (;;) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_ready.wait(lk, [&] { return s->stop || !s->ready.empty(); });
            if (s->stop && s->ready.empty()) return;
            while (!s->ready.empty() && (int)batch.size() < s->opts.max_batch) {
                batch.push_back(s->ready.front());
                s->ready.pop_front();
            }
        }
        std::vector<pne_terms *> terms;
        for (Request *r : batch) terms.push_back(r->terms);
        pne_batch_opts bo{s->opts.warps_per_block, s->opts.blocks_per_sm, 0};
        pne_batch *b = nullptr;
        pne_status rc = pne_batch_create(s->ctx, (int32_t)terms.size(), terms.data(), (pne_dtype)s->opts.dtype, &bo,
                                         s->launch_stream, &b);
        if (rc == PNE_EINVAL) {            // the shape does not fit these clusters: smallest shape
            pne_batch_opts small{1, 1, 0};
            rc = pne_batch_create(s->ctx, (int32_t)terms.size(), terms.data(), (pne_dtype)s->opts.dtype, &small,
                                  s->launch_stream, &b);
        }
        std::vector<pne_result> res(batch.size());
        if (rc == PNE_OK) rc = pne_batch_run(s->ctx, b, s->launch_stream, res.data());
        if (b) pne_batch_destroy(b);
        // a failed create or run may leave work queued for these requests:
        // let it finish before their buffers go (their release is fenced
        // behind the launch stream anyway; this keeps a failure contained)
        if (rc != PNE_OK) cudaStreamSynchronize(s->launch_stream);
        for (Request *r : batch) release(r);
        std::unique_lock<std::mutex> lk(s->mu);
        for (size_t i = 0; i < batch.size(); ++i) {
            Request *r = batch[i];
            if (rc == PNE_OK) r->result = res[i];
            r->info.batch_size = (int32_t)batch.size();
            finish_locked(s, r, rc);
        }
        s->cv_admit.notify_all();
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

pne_status pne_server_create(pne_ctx *ctx, const pne_server_opts *opts, pne_server **out)
{
    if (!ctx || !out) return PNE_EINVAL;
    *out = nullptr;
    pne_server *s = new pne_server();
    s->ctx = ctx;
    if (opts) s->opts = *opts;
    if (s->opts.device_budget_bytes == 0) s->opts.device_budget_bytes = 8ull << 30;
    if (s->opts.max_inflight <= 0) s->opts.max_inflight = 256;
    if (s->opts.n_prep_streams <= 0) s->opts.n_prep_streams = 4;
    if (s->opts.max_batch <= 0) s->opts.max_batch = 256;
    if (s->opts.warps_per_block <= 0) s->opts.warps_per_block = 4;
    if (s->opts.blocks_per_sm <= 0) s->opts.blocks_per_sm = 2;
    if (s->opts.dtype < PNE_F64 || s->opts.dtype > PNE_BF16) { delete s; return PNE_EINVAL; }
    s->t0 = std::chrono::steady_clock::now();
    cudaSetDevice(ctx->device);
    s->streams.resize(s->opts.n_prep_streams);
    for (auto &st : s->streams)
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) { delete s; return PNE_ECUDA; }
    if (cudaStreamCreateWithFlags(&s->launch_stream, cudaStreamNonBlocking) != cudaSuccess) { delete s; return PNE_ECUDA; }
    for (int w = 0; w < s->opts.n_prep_streams; ++w) s->prep.emplace_back(prep_loop, s, w);
    s->launcher = std::thread(launch_loop, s);
    *out = s;
    return PNE_OK;
}

pne_status pne_server_submit(pne_server *s, const pne_network *net, int32_t max_order, uint64_t *id)
{
    if (!s || !net || !id || net->n_batch != 1 || net->data_on_device || !net->data || net->n_sites < 1 ||
        max_order < 0 || max_order > PNE_MAX_ORDER)
        return PNE_EINVAL;
    for (int b = 0; b < net->n_bonds; ++b)
        if (net->bond_site[2 * b + 1] < 0) return PNE_EINVAL;     // open indices are not served
    Request *r = new Request();
    r->n_sites = net->n_sites; r->n_bonds = net->n_bonds; r->K = max_order;
    r->bond_site.assign(net->bond_site, net->bond_site + 2 * net->n_bonds);
    r->bond_dim.assign(net->bond_dim, net->bond_dim + net->n_bonds);
    r->site_ptr.assign(net->site_ptr, net->site_ptr + net->n_sites + 1);
    r->site_bonds.assign(net->site_bonds, net->site_bonds + net->site_ptr[net->n_sites]);
    r->data_off.assign(net->data_off, net->data_off + net->n_sites + 1);
    r->data.assign(net->data, net->data + net->data_off[net->n_sites]);
    r->est_bytes = estimate_bytes(s, *r);
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->info.t_arrival = s->now();
    r->info.device_bytes = r->est_bytes;
    s->all[r->id] = r;
    s->arrivals.push_back(r);
    s->outstanding += 1;
    *id = r->id;
    s->cv_admit.notify_all();
    return PNE_OK;
}

pne_status pne_server_poll(pne_server *s, uint64_t id, pne_result *out, pne_request_info *info)
{
    if (!s) return PNE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return PNE_EINVAL;
    Request *r = it->second;
    if (!r->done) return PNE_EBUSY;
    if (out) *out = r->result;
    if (info) *info = r->info;
    const pne_status st = r->status;
    s->all.erase(it);
    delete r;
    return st;
}

pne_status pne_server_drain(pne_server *s)
{
    if (!s) return PNE_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
    return PNE_OK;
}

pne_status pne_server_stats(pne_server *s, uint64_t *peak_inflight_bytes, double *now)
{
    if (!s) return PNE_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (peak_inflight_bytes) *peak_inflight_bytes = s->peak_bytes;
    if (now) *now = s->now();
    return PNE_OK;
}

const char *pne_server_first_error(pne_server *s)
{
    if (!s) return "";
    std::lock_guard<std::mutex> lk(s->mu);
    return s->first_error.c_str();
}

void pne_server_destroy(pne_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_admit.notify_all();
    s->cv_ready.notify_all();
    for (auto &t : s->prep) t.join();
    if (s->launcher.joinable()) s->launcher.join();
    for (auto &kv : s->all) { release(kv.second); delete kv.second; }
    for (auto st : s->streams) cudaStreamDestroy(st);
    if (s->launch_stream) cudaStreamDestroy(s->launch_stream);
    delete s;
}

}  // extern "C"
