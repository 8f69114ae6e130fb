// Host side of libpne: the C ABI of include/pne.h.
//
// Validation of the network, geometry tables (leg positions, incoming-message
// slots, row-major and excitation-blocked offsets), device memory through the
// context's allocator, the enumeration cache, and the final FP64 assembly of
// each result (Z_K = Z_ref * sum_k c_k, Sec. II.B truncation of Eq. A4).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <limits>
#include <map>
#include <string>
#include <vector>

#include "pne_internal.h"

namespace {
thread_local std::string g_last_error;
}

namespace pne {

void set_error(pne_ctx *ctx, pne_status st, const std::string &msg)
{
    (void)ctx;
    g_last_error = std::string("pne status ") + std::to_string((int)st) + ": " + msg;
}

pne_status dev_alloc(pne_ctx *ctx, DevBuf &b, size_t bytes, cudaStream_t s)
{
    if (bytes < 16) bytes = 16;
    b.bytes = bytes;
    if (ctx->alloc) {
        b.ptr = ctx->alloc(bytes, (void *)s, ctx->alloc_user);
        if (!b.ptr) { set_error(ctx, PNE_ENOMEM, "allocator callback returned NULL"); return PNE_ENOMEM; }
        return PNE_OK;
    }
    cudaError_t e = cudaMallocAsync(&b.ptr, bytes, s);
    if (e != cudaSuccess) {
        b.ptr = nullptr;
        set_error(ctx, PNE_ENOMEM, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
        return PNE_ENOMEM;
    }
    return PNE_OK;
}

int64_t *pinned_i64(pne_ctx *ctx, size_t n)
{
    (void)ctx;
    thread_local int64_t *buf = nullptr;
    thread_local size_t cap = 0;
    thread_local int64_t fallback[64];          // pageable, if pinned memory is unavailable
    if (n > cap) {
        if (buf) cudaFreeHost(buf);
        cap = n < 64 ? 64 : n;
        if (cudaMallocHost((void **)&buf, cap * 8) != cudaSuccess) { buf = nullptr; cap = 0; }
    }
    return buf ? buf : (n <= 64 ? fallback : nullptr);
}

namespace {
struct HostStage {
    char *buf = nullptr;
    size_t cap = 0, used = 0;
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> marks;   // last copy queued per stream
};
HostStage &host_stage()
{
    thread_local HostStage h;
    return h;
}
}  // namespace

pne_status upload(pne_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s)
{
    if (bytes == 0) return PNE_OK;
    HostStage &h = host_stage();
    const size_t need = (bytes + 255) & ~size_t(255);
    if (h.used + need > h.cap) {
        // recycle the region once every copy out of it has completed
        for (auto &m : h.marks) {
            cudaEventSynchronize(m.second);
            cudaEventDestroy(m.second);
        }
        h.marks.clear();
        h.used = 0;
        if (need > h.cap) {
            if (h.buf) cudaFreeHost(h.buf);
            h.cap = std::max(need, std::max<size_t>(2 * h.cap, size_t(1) << 20));
            if (cudaMallocHost((void **)&h.buf, h.cap) != cudaSuccess) { h.buf = nullptr; h.cap = 0; }
        }
    }
    if (!h.buf) {                                   // no pinned memory: a pageable copy
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return PNE_OK;
    }
    char *stage = h.buf + h.used;
    std::memcpy(stage, src, bytes);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyHostToDevice, s));
    h.used += need;
    cudaEvent_t ev = nullptr;
    for (auto &m : h.marks)
        if (m.first == s) ev = m.second;
    if (!ev) {
        PNE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        h.marks.push_back({s, ev});
    }
    PNE_CUDA_TRY(ctx, cudaEventRecord(ev, s));
    return PNE_OK;
}

void *pinned_slot(int slot, size_t bytes)
{
    thread_local void *buf[kPinnedSlots] = {};
    thread_local size_t cap[kPinnedSlots] = {};
    if (slot < 0 || slot >= kPinnedSlots) return nullptr;
    if (bytes > cap[slot]) {
        if (buf[slot]) cudaFreeHost(buf[slot]);
        cap[slot] = std::max<size_t>(bytes, 4096);
        if (cudaMallocHost(&buf[slot], cap[slot]) != cudaSuccess) { buf[slot] = nullptr; cap[slot] = 0; }
    }
    return buf[slot];
}

void *take_pinned(pne_ctx *ctx, size_t bytes, size_t *got)
{
    {
        std::lock_guard<std::mutex> lk(ctx->pinned_mu);
        size_t best = ctx->pinned_pool.size();
        for (size_t i = 0; i < ctx->pinned_pool.size(); ++i)
            if (ctx->pinned_pool[i].second >= bytes &&
                (best == ctx->pinned_pool.size() || ctx->pinned_pool[i].second < ctx->pinned_pool[best].second))
                best = i;
        if (best < ctx->pinned_pool.size()) {
            void *p = ctx->pinned_pool[best].first;
            *got = ctx->pinned_pool[best].second;
            ctx->pinned_pool.erase(ctx->pinned_pool.begin() + best);
            return p;
        }
    }
    const size_t cap = std::max<size_t>(bytes, 64 * 1024);
    void *p = nullptr;
    if (cudaMallocHost(&p, cap) != cudaSuccess) return nullptr;
    *got = cap;
    return p;
}

void give_pinned(pne_ctx *ctx, void *p, size_t bytes)
{
    if (!p) return;
    std::lock_guard<std::mutex> lk(ctx->pinned_mu);
    ctx->pinned_pool.push_back({p, bytes});
}

void dev_free(pne_ctx *ctx, DevBuf &b, cudaStream_t s)
{
    if (!b.ptr) return;
    if (ctx->free_fn) ctx->free_fn(b.ptr, b.bytes, (void *)s, ctx->alloc_user);
    else cudaFreeAsync(b.ptr, s);
    b.ptr = nullptr;
    b.bytes = 0;
}

cudaError_t grant_dynamic_smem(const void *func, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    static std::mutex mu;
    static std::map<const void *, size_t> granted;
    std::lock_guard<std::mutex> lk(mu);
    size_t &g = granted[func];
    if (bytes <= g) return cudaSuccess;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g = bytes;
    return e;
}

cudaEvent_t take_event(pne_ctx *ctx)
{
    {
        std::lock_guard<std::mutex> lk(ctx->event_mu);
        if (!ctx->event_pool.empty()) {
            cudaEvent_t ev = ctx->event_pool.back();
            ctx->event_pool.pop_back();
            return ev;
        }
    }
    cudaEvent_t ev = nullptr;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    return ev;
}

void give_event(pne_ctx *ctx, cudaEvent_t ev)
{
    if (!ev) return;
    std::lock_guard<std::mutex> lk(ctx->event_mu);
    ctx->event_pool.push_back(ev);
}

void UseFence::note(pne_ctx *ctx, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(mu);
    for (auto &u : uses)
        if (u.first == s) { cudaEventRecord(u.second, s); return; }
    cudaEvent_t ev = take_event(ctx);
    if (!ev) {
        // no event: wait here for the stream's queued work instead
        cudaStreamSynchronize(s);
        return;
    }
    cudaEventRecord(ev, s);
    uses.push_back({s, ev});
}

bool UseFence::join(cudaStream_t target)
{
    std::lock_guard<std::mutex> lk(mu);
    bool ok = true;
    for (auto &u : uses)
        if (cudaStreamWaitEvent(target, u.second, 0) != cudaSuccess) ok = false;
    return ok;
}

void UseFence::release(pne_ctx *ctx)
{
    std::lock_guard<std::mutex> lk(mu);
    for (auto &u : uses) give_event(ctx, u.second);
    uses.clear();
}

ProfScope::ProfScope(pne_ctx *c, cudaStream_t st, const char *n) : ctx(c), s(st), name(n)
{
    if (!ctx || !ctx->prof.on) return;
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    auto take = [&]() {
        cudaEvent_t e;
        if (!ctx->prof.pool.empty()) { e = ctx->prof.pool.back(); ctx->prof.pool.pop_back(); }
        else cudaEventCreate(&e);
        return e;
    };
    a = take();
    b = take();
    cudaEventRecord(a, s);
}

ProfScope::~ProfScope()
{
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    ctx->prof.pending.push_back({name, a, b, s});
}

HostScope::HostScope(pne_ctx *c, const char *n) : ctx(c), name(n)
{
    if (!ctx || !ctx->prof.on) return;
    t0 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

HostScope::~HostScope() { stop(); }

void HostScope::stop()
{
    if (t0 < 0.0) return;
    const double t1 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    auto &e = ctx->prof.acc[std::string("host:") + name];
    e.first += 1;
    e.second += t1 - t0;
    if (ctx->prof.trace && ctx->prof.host_trace.size() < kTraceMax)
        ctx->prof.host_trace.push_back({name, t0 - ctx->prof.host_base, t1 - ctx->prof.host_base});
    t0 = -1.0;
}

EnumRecord::~EnumRecord()
{
    if (!ctx) return;
    // released after every stream that used the record (the search and shape
    // streams, the contractions and sums of every terms handle) reaches the
    // point where it stopped using it
    cudaStream_t rs = ctx->release_stream;
    if (!uses.join(rs)) { cudaDeviceSynchronize(); rs = nullptr; }
    uses.release(ctx);
    dev_free(ctx, cl_edges, rs);
    dev_free(ctx, cl_verts, rs);
    dev_free(ctx, cl_size, rs);
    for (auto &L : levels) dev_free(ctx, L.idx, rs);
    dev_free(ctx, shape_of, rs);
    dev_free(ctx, perm, rs);
    dev_free(ctx, plans, rs);
    dev_free(ctx, plan_steps, rs);
    dev_free(ctx, ops, rs);
    dev_free(ctx, op_off, rs);
    dev_free(ctx, step_off, rs);
    dev_free(ctx, step_site, rs);
    dev_free(ctx, vgeo.storage, rs);
    dev_free(ctx, sum_desc, rs);
}

namespace {

uint64_t fnv(uint64_t h, const void *p, size_t n)
{
    const unsigned char *c = (const unsigned char *)p;
    for (size_t i = 0; i < n; ++i) { h ^= c[i]; h *= 1099511628211ull; }
    return h;
}

}  // namespace

// Derived tables of a geometry given bond_site, bond_dim, site_ptr, site_bonds.
pne_status finish_geometry(pne_ctx *ctx, Geometry &g, cudaStream_t s)
{
    HostScope hs__(ctx, "geometry");
    const int N = g.n_sites, M = g.n_bonds;
    g.n_legs = g.site_ptr[N];
    g.bond_leg.assign(2 * M, -1);
    g.max_deg = 0; g.max_dim = 0;
    for (int v = 0; v < N; ++v) {
        const int k = g.site_ptr[v + 1] - g.site_ptr[v];
        g.max_deg = std::max(g.max_deg, k);
        for (int i = 0; i < k; ++i) {
            const int b = g.site_bonds[g.site_ptr[v] + i];
            const int side = (g.bond_site[2 * b] == v) ? 0 : 1;
            g.bond_leg[2 * b + side] = i;
        }
    }
    for (int b = 0; b < M; ++b) g.max_dim = std::max(g.max_dim, g.bond_dim[b]);
    g.inc_slot.assign(g.n_legs, 0);
    for (int v = 0; v < N; ++v)
        for (int i = g.site_ptr[v]; i < g.site_ptr[v + 1]; ++i) {
            const int b = g.site_bonds[i];
            const int s0 = g.bond_site[2 * b], s1 = g.bond_site[2 * b + 1];
            if (s1 < 0) { g.inc_slot[i] = i; continue; }         // boundary reflection
            const int u = (s0 == v) ? s1 : s0, side = (s0 == v) ? 1 : 0;
            g.inc_slot[i] = g.site_ptr[u] + g.bond_leg[2 * b + side];
        }
    g.tens_off.assign(N + 1, 0);
    g.blk_off.assign((size_t)N * kBlkStride, 0);
    for (int v = 0; v < N; ++v) {
        const int k = g.site_ptr[v + 1] - g.site_ptr[v];
        int64_t n = 1;
        int q[kMaxDeg];
        for (int i = 0; i < k; ++i) { const int d = g.bond_dim[g.site_bonds[g.site_ptr[v] + i]]; n *= d; q[i] = d - 1; }
        g.tens_off[v + 1] = g.tens_off[v] + n;
        int32_t off = 0;
        for (int m = 0; m < (1 << k); ++m) {
            g.blk_off[(size_t)v * kBlkStride + m] = off;
            int32_t sz = 1;
            for (int i = 0; i < k; ++i) if (m >> i & 1) sz *= q[i];
            off += sz;
        }
    }
    // greedy colouring in site order over the closed bonds: every site takes the
    // smallest colour none of its earlier neighbours has (a checkerboard on
    // the square and cubic lattices)
    {
        std::vector<int32_t> col(N, -1);
        std::vector<char> used;
        int nc = 0;
        for (int v = 0; v < N; ++v) {
            used.assign(nc + 1, 0);
            for (int i = g.site_ptr[v]; i < g.site_ptr[v + 1]; ++i) {
                const int b = g.site_bonds[i];
                const int s0 = g.bond_site[2 * b], s1 = g.bond_site[2 * b + 1];
                if (s1 < 0) continue;
                const int u = (s0 == v) ? s1 : s0;
                if (col[u] >= 0) used[col[u]] = 1;
            }
            int c = 0;
            while (used[c]) ++c;
            col[v] = c;
            nc = std::max(nc, c + 1);
        }
        g.n_colors = nc;
        g.color_ptr.assign(nc + 1, 0);
        for (int v = 0; v < N; ++v) ++g.color_ptr[col[v] + 1];
        for (int c = 0; c < nc; ++c) g.color_ptr[c + 1] += g.color_ptr[c];
        g.color_sites.assign(N, 0);
        std::vector<int32_t> fill(g.color_ptr.begin(), g.color_ptr.end() - 1);
        for (int v = 0; v < N; ++v) g.color_sites[fill[col[v]]++] = v;
        // within a colour (sites updated independently, in any order) by leg
        // count, then id: the float-float sweeps take neighbouring entries
        // two at a time, and sites of one leg count share a code path
        for (int c = 0; c < nc; ++c)
            std::stable_sort(g.color_sites.begin() + g.color_ptr[c], g.color_sites.begin() + g.color_ptr[c + 1],
                             [&](int a, int b) {
                                 return g.site_ptr[a + 1] - g.site_ptr[a] < g.site_ptr[b + 1] - g.site_ptr[b];
                             });
    }
    g.site_nbr.assign(2 * g.site_bonds.size(), -1);
    for (int v = 0; v < N; ++v)
        for (int i = g.site_ptr[v]; i < g.site_ptr[v + 1]; ++i) {
            const int b = g.site_bonds[i];
            g.site_nbr[2 * i] = b;
            g.site_nbr[2 * i + 1] = g.bond_site[2 * b] == v ? g.bond_site[2 * b + 1] : g.bond_site[2 * b];
        }
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, &N, sizeof N);
    h = fnv(h, g.bond_site.data(), g.bond_site.size() * 4);
    h = fnv(h, g.bond_dim.data(), g.bond_dim.size() * 4);
    g.hash = h;
    // one device buffer for every table
    const size_t n_i32 = g.bond_site.size() + g.bond_dim.size() + g.site_ptr.size() + g.site_bonds.size() +
                         g.bond_leg.size() + g.inc_slot.size() + g.blk_off.size() + g.color_ptr.size() +
                         g.color_sites.size() + g.site_nbr.size();
    const size_t bytes = g.tens_off.size() * 8 + n_i32 * 4 + 64;
    pne_status st = dev_alloc(ctx, g.storage, bytes, s);
    if (st) return st;
    std::vector<char> host(bytes, 0);
    size_t off = 0;
    auto put = [&](const void *src, size_t nb) { size_t o = off; std::memcpy(host.data() + off, src, nb); off += nb; return o; };
    const size_t o_tens = put(g.tens_off.data(), g.tens_off.size() * 8);
    const size_t o_nbr = put(g.site_nbr.data(), g.site_nbr.size() * 4);      // 8-byte aligned pairs
    const size_t o_bs = put(g.bond_site.data(), g.bond_site.size() * 4);
    const size_t o_bd = put(g.bond_dim.data(), g.bond_dim.size() * 4);
    const size_t o_sp = put(g.site_ptr.data(), g.site_ptr.size() * 4);
    const size_t o_sb = put(g.site_bonds.data(), g.site_bonds.size() * 4);
    const size_t o_bl = put(g.bond_leg.data(), g.bond_leg.size() * 4);
    const size_t o_is = put(g.inc_slot.data(), g.inc_slot.size() * 4);
    const size_t o_bo = put(g.blk_off.data(), g.blk_off.size() * 4);
    const size_t o_cp = put(g.color_ptr.data(), g.color_ptr.size() * 4);
    const size_t o_cs = put(g.color_sites.data(), g.color_sites.size() * 4);
    char *d = (char *)g.storage.ptr;
    g.d_tens_off = (int64_t *)(d + o_tens);
    g.d_site_nbr = (int2 *)(d + o_nbr);
    g.d_bond_site = (int32_t *)(d + o_bs);
    g.d_bond_dim = (int32_t *)(d + o_bd);
    g.d_site_ptr = (int32_t *)(d + o_sp);
    g.d_site_bonds = (int32_t *)(d + o_sb);
    g.d_bond_leg = (int32_t *)(d + o_bl);
    g.d_inc_slot = (int32_t *)(d + o_is);
    g.d_blk_off = (int32_t *)(d + o_bo);
    g.d_color_ptr = (int32_t *)(d + o_cp);
    g.d_color_sites = (int32_t *)(d + o_cs);
    return upload(ctx, g.storage.ptr, host.data(), bytes, s);
}

namespace {

pne_status validate(pne_ctx *ctx, const pne_network *n, int max_dim = kMaxDim, int64_t max_size = 4096)
{
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    if (!n || n->n_sites < 1 || n->n_bonds < 0) return bad("empty or malformed network");
    if (!n->bond_site || !n->bond_dim || !n->site_ptr || !n->site_bonds || !n->data || !n->data_off)
        return bad("null array in pne_network");
    if (n->n_batch < 1) return bad("n_batch must be >= 1");
    const int N = n->n_sites, M = n->n_bonds;
    std::vector<int> seen(M, 0);
    for (int b = 0; b < M; ++b) {
        const int s0 = n->bond_site[2 * b], s1 = n->bond_site[2 * b + 1];
        if (s0 < 0 || s0 >= N || s1 >= N || s1 < -1 || s0 == s1) return bad("bond " + std::to_string(b) + " has invalid sites");
        if (n->bond_dim[b] < 2 || n->bond_dim[b] > max_dim)
            return bad("bond dimension must be in 2.." + std::to_string(max_dim));
    }
    if (n->site_ptr[0] != 0) return bad("site_ptr[0] must be 0");
    for (int v = 0; v < N; ++v) {
        const int a = n->site_ptr[v], e = n->site_ptr[v + 1];
        if (e < a || e - a > kMaxDeg) return bad("site degree must be in 0..6");
        int64_t size = 1;
        for (int i = a; i < e; ++i) {
            const int b = n->site_bonds[i];
            if (b < 0 || b >= M) return bad("site_bonds out of range");
            if (i > a && n->site_bonds[i - 1] >= b) return bad("legs must be in ascending bond id");
            if (n->bond_site[2 * b] != v && n->bond_site[2 * b + 1] != v) return bad("leg not incident to its site");
            seen[b]++;
            size *= n->bond_dim[b];
        }
        if (n->data_off[v + 1] - n->data_off[v] != size) return bad("data_off inconsistent with leg dimensions");
        if (size > max_size) return bad("site tensor larger than " + std::to_string(max_size) + " entries");
    }
    if (n->data_off[0] != 0) return bad("data_off[0] must be 0");
    for (int b = 0; b < M; ++b) {
        const int want = (n->bond_site[2 * b + 1] < 0) ? 1 : 2;
        if (seen[b] != want) return bad("bond " + std::to_string(b) + " not listed at both of its sites");
    }
    return PNE_OK;
}

double gamma_n(int n, double u) { return (n * u) / (1.0 - n * u); }

}  // namespace

void finalize_result(pne_result &r, int K, int mode, int dtype, const double *c, const double *abs_c,
                     const double *vac, uint64_t n_terms, uint64_t n_clusters, int bp_iters, double bp_residual)
{
    static const double unit[4] = {0x1p-53, 0x1p-24, 0x1p-11, 0x1p-8};
    const double u = unit[dtype < 0 ? 0 : dtype];
    // first-order rounding count per term: every site factor and every
    // intermediate of a cluster contraction is rounded once in the working
    // dtype (at most 2 (K + 1) roundings along a term's product)
    const int nops = 2 * (K + 1);
    std::memset(&r, 0, sizeof r);
    const double lz = vac[0], sz = vac[1];
    const int nzero = (int)vac[2];
    r.n_orders = K + 1;
    for (int k = 0; k <= K; ++k) { r.c[k] = c[k]; r.abs_c[k] = abs_c[k]; }
    if (mode == PNE_MODE_LOOP && nzero == 0) { r.c[0] += 1.0; r.abs_c[0] += 1.0; }
    double sum = 0.0, comp = 0.0, asum = 0.0;            // Neumaier over orders
    for (int k = 0; k <= K; ++k) {
        const double x = r.c[k], tt = sum + x;
        comp += (std::fabs(sum) >= std::fabs(x)) ? (sum - tt) + x : (x - tt) + sum;
        sum = tt;
        asum += r.abs_c[k];
    }
    sum += comp;
    r.log_abs_zref = lz;
    r.sign_zref = sz < 0 ? -1 : 1;
    r.n_zero_sites = nzero;
    r.sign = (sum < 0 ? -1 : 1) * r.sign_zref;
    r.log_abs = (sum != 0.0) ? lz + std::log(std::fabs(sum)) : -std::numeric_limits<double>::infinity();
    r.value = (sum == 0.0) ? 0.0 : (r.log_abs > 709.7 ? r.sign * std::numeric_limits<double>::infinity()
                                                       : r.sign * std::exp(r.log_abs));
    if (nzero == 0 && r.c[0] != 0.0) {                    // truncated power-series logarithm
        double cc[kMaxOrder + 1], l[kMaxOrder + 1];
        for (int k = 0; k <= K; ++k) { cc[k] = r.c[k] / r.c[0]; l[k] = 0.0; }
        double ls = 0.0;
        for (int k = 1; k <= K; ++k) {
            double acc = k * cc[k];
            for (int j = 1; j < k; ++j) acc -= j * l[j] * cc[k - j];
            l[k] = acc / k;
            ls += l[k];
        }
        r.log_series = lz + std::log(std::fabs(r.c[0])) + ls;
    } else {
        r.log_series = std::numeric_limits<double>::quiet_NaN();
    }
    // Only cluster values carry the working dtype's rounding: the empty term
    // (exactly 1 in FP64 when no site has z_v == 0) does not, so it is left
    // out of the absolute sum the dtype's bound multiplies.  The FP64 products
    // and sums add at most (K + 2 + log2 of the term count) roundings of 2^-53
    // on every term.
    const double exact = (nzero == 0) ? 1.0 : 0.0;
    const double cl_abs = std::max(0.0, asum - exact);
    const int n64 = K + 2 + (int)std::ceil(std::log2((double)std::max<uint64_t>(n_terms, 2)));
    r.err_bound = (sum != 0.0) ? (gamma_n(nops, u) * cl_abs + gamma_n(n64, 0x1p-53) * asum) / std::fabs(sum)
                               : std::numeric_limits<double>::infinity();
    r.n_terms = n_terms;
    r.n_clusters = n_clusters;
    r.bp_iters = bp_iters;
    r.bp_residual = bp_residual;
}

// The combinatorial form's result (Eq. A6 without the residue): the sub-network
// sums c_k (k = |x|) enter with the sign (-1)^{k+1}.  Every sub-network is an
// exact contraction of at most all N sites, so a product path rounds at most
// 2 N times in the working dtype.
void finalize_comb_result(pne_result &r, int M, int dtype, const double *c, const double *abs_c, const double *vac,
                          uint64_t n_terms, uint64_t n_clusters, int n_sites, int bp_iters, double bp_residual)
{
    static const double unit[4] = {0x1p-53, 0x1p-24, 0x1p-11, 0x1p-8};
    const double u = unit[dtype < 0 ? 0 : dtype];
    std::memset(&r, 0, sizeof r);
    const double lz = vac[0], sz = vac[1];
    r.n_orders = M + 1;
    double sum = 0.0, comp = 0.0, asum = 0.0;            // Neumaier over |x|
    for (int k = 0; k <= M; ++k) {
        r.c[k] = c[k];
        r.abs_c[k] = abs_c[k];
        const double x = (k % 2 == 1) ? c[k] : -c[k], tt = sum + x;
        if (k == 0) continue;
        comp += (std::fabs(sum) >= std::fabs(x)) ? (sum - tt) + x : (x - tt) + sum;
        sum = tt;
        asum += abs_c[k];
    }
    sum += comp;
    r.log_abs_zref = lz;
    r.sign_zref = sz < 0 ? -1 : 1;
    r.n_zero_sites = (int)vac[2];
    r.sign = (sum < 0 ? -1 : 1) * r.sign_zref;
    r.log_abs = (sum != 0.0) ? lz + std::log(std::fabs(sum)) : -std::numeric_limits<double>::infinity();
    r.value = (sum == 0.0) ? 0.0 : (r.log_abs > 709.7 ? r.sign * std::numeric_limits<double>::infinity()
                                                       : r.sign * std::exp(r.log_abs));
    r.log_series = std::numeric_limits<double>::quiet_NaN();
    const int n64 = M + 2 + (int)std::ceil(std::log2((double)std::max<uint64_t>(n_terms, 2)));
    r.err_bound = (sum != 0.0) ? (gamma_n(2 * n_sites, u) + gamma_n(n64, 0x1p-53)) * asum / std::fabs(sum)
                               : std::numeric_limits<double>::infinity();
    r.n_terms = n_terms;
    r.n_clusters = n_clusters;
    r.bp_iters = bp_iters;
    r.bp_residual = bp_residual;
}

// 64-bit hash of the raw geometry arrays (multiply-rotate over 32-bit words)
uint64_t geometry_key(const pne_network *net)
{
    uint64_t h = 0x9E3779B97F4A7C15ull ^ ((uint64_t)(uint32_t)net->n_sites << 32 | (uint32_t)net->n_bonds);
    auto mix = [&h](const int32_t *a, size_t n) {
        for (size_t i = 0; i < n; ++i) {
            h ^= (uint32_t)a[i];
            h *= 0xBF58476D1CE4E5B9ull;
            h ^= h >> 31;
        }
    };
    mix(net->bond_site, 2 * (size_t)net->n_bonds);
    mix(net->bond_dim, (size_t)net->n_bonds);
    mix(net->site_ptr, (size_t)net->n_sites + 1);
    mix(net->site_bonds, (size_t)net->site_ptr[net->n_sites]);
    return h;
}

bool same_geometry(const GeomPair &g, const pne_network *net)
{
    const Geometry &f = g.full;
    const int N = net->n_sites, M = net->n_bonds;
    return f.n_sites == N && f.n_bonds == M && (int)f.site_bonds.size() == net->site_ptr[N] &&
           std::equal(f.bond_site.begin(), f.bond_site.end(), net->bond_site) &&
           std::equal(f.bond_dim.begin(), f.bond_dim.end(), net->bond_dim) &&
           std::equal(f.site_ptr.begin(), f.site_ptr.end(), net->site_ptr) &&
           std::equal(f.site_bonds.begin(), f.site_bonds.end(), net->site_bonds);
}

constexpr size_t kGeomCacheMax = 256;   // geometries kept per context

// The full and closed geometry of a (validated) network: from the context's
// cache when the same arrays were seen before, else built, uploaded on `s`
// and cached.
pne_status build_geometry(pne_ctx *ctx, const pne_network *net, GeomPair &gpr, cudaStream_t s);

pne_status get_geometry(pne_ctx *ctx, const pne_network *net, cudaStream_t s, std::shared_ptr<GeomPair> &out)
{
    HostScope hs__(ctx, "geometry");
    const uint64_t key = geometry_key(net);
    {
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        auto it = ctx->geom_cache.find(key);
        if (it != ctx->geom_cache.end())
            for (auto &g : it->second)
                if (same_geometry(*g, net)) {
                    // the device copies may have been queued on another stream
                    if (g->ready) PNE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, g->ready, 0));
                    out = g;
                    return PNE_OK;
                }
    }
    auto gp = std::make_shared<GeomPair>();
    gp->ctx = ctx;
    gp->key = key;
    pne_status st = build_geometry(ctx, net, *gp, s);
    // the uploads (and, on failure, whatever was queued) are on `s`: the
    // geometry's memory is released only after them
    gp->uses.note(ctx, s);
    if (st) return st;
    PNE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&gp->ready, cudaEventDisableTiming));
    PNE_CUDA_TRY(ctx, cudaEventRecord(gp->ready, s));
    {
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        size_t n = 0;
        for (auto &kv : ctx->geom_cache) n += kv.second.size();
        if (n < kGeomCacheMax) ctx->geom_cache[key].push_back(gp);
    }
    out = gp;
    return PNE_OK;
}

// Host tables and device copies (queued on `s`) of a validated network.
pne_status build_geometry(pne_ctx *ctx, const pne_network *net, GeomPair &gpr, cudaStream_t s)
{
    GeomPair *gp = &gpr;
    const int N = net->n_sites, M = net->n_bonds;
    Geometry &f = gp->full;
    f.n_sites = N; f.n_bonds = M;
    f.bond_site.assign(net->bond_site, net->bond_site + 2 * M);
    f.bond_dim.assign(net->bond_dim, net->bond_dim + M);
    f.site_ptr.assign(net->site_ptr, net->site_ptr + N + 1);
    f.site_bonds.assign(net->site_bonds, net->site_bonds + net->site_ptr[N]);
    // closed geometry: open bonds removed, remaining bonds renumbered in order
    gp->closed_of_full.assign(M, -1);
    Geometry &c = gp->closed;
    c.n_sites = N;
    int mc = 0;
    for (int b = 0; b < M; ++b) {
        if (f.bond_site[2 * b + 1] < 0) { gp->open_bonds.push_back(b); gp->open_dims.push_back(f.bond_dim[b]); continue; }
        gp->closed_of_full[b] = mc++;
        c.bond_site.push_back(f.bond_site[2 * b]); c.bond_site.push_back(f.bond_site[2 * b + 1]);
        c.bond_dim.push_back(f.bond_dim[b]);
    }
    c.n_bonds = mc;
    c.site_ptr.assign(N + 1, 0);
    for (int v = 0; v < N; ++v) {
        for (int i = f.site_ptr[v]; i < f.site_ptr[v + 1]; ++i) {
            const int cb = gp->closed_of_full[f.site_bonds[i]];
            if (cb >= 0) c.site_bonds.push_back(cb);
        }
        c.site_ptr[v + 1] = (int32_t)c.site_bonds.size();
    }
    pne_status st;
    if ((st = finish_geometry(ctx, f, s)) || (st = finish_geometry(ctx, c, s))) return st;
    {
        // gauge-transform table: open position per full bond, then the open dims
        for (int v = 0; v < N; ++v) {
            int n = 1;
            for (int i = f.site_ptr[v]; i < f.site_ptr[v + 1]; ++i) n *= f.bond_dim[f.site_bonds[i]];
            gp->gauge_nmax = std::max(gp->gauge_nmax, n);
        }
        std::vector<int32_t> h(M, -1);
        for (size_t q = 0; q < gp->open_bonds.size(); ++q) h[gp->open_bonds[q]] = (int32_t)q;
        h.insert(h.end(), gp->open_dims.begin(), gp->open_dims.end());
        h.push_back(0);
        if ((st = dev_alloc(ctx, gp->gauge_tab, h.size() * 4, s)) ||
            (st = upload(ctx, gp->gauge_tab.ptr, h.data(), h.size() * 4, s)))
            return st;
    }
    return PNE_OK;
}

GeomPair::~GeomPair()
{
    if (ready) cudaEventDestroy(ready);
    if (!ctx) return;
    // after every partition that used it (their streams may be gone by now)
    cudaStream_t rs = ctx->release_stream;
    if (!uses.join(rs)) { cudaDeviceSynchronize(); rs = nullptr; }
    uses.release(ctx);
    dev_free(ctx, full.storage, rs);
    dev_free(ctx, closed.storage, rs);
    dev_free(ctx, gauge_tab, rs);
}

// A validated network's geometry through the context's cache (for the other
// translation units' entry points).
pne_status geometry_for(pne_ctx *ctx, const pne_network *net, cudaStream_t s, std::shared_ptr<GeomPair> &out,
                        int max_dim, int64_t max_size)
{
    pne_status st = validate(ctx, net, max_dim, max_size);
    if (st) return st;
    return get_geometry(ctx, net, s, out);
}

pne_status partition_record(pne_ctx *ctx, pne_partition *p, const char *rec)
{
    const size_t B = p->n_sets;
    const int32_t *flags = (const int32_t *)(rec + B * 8);
    std::memcpy(p->bp_residual.data(), rec, B * 8);
    std::memcpy(p->bp_iters.data(), rec + B * 8 + 16, B * 4);
    p->rec_pending = false;
    if (flags[0] || flags[2]) { set_error(ctx, PNE_ETIMEOUT, "grid barrier timed out in BP"); return PNE_ETIMEOUT; }
    if (flags[1] || flags[3]) { set_error(ctx, PNE_EDEGENERATE, "zero message or zero message overlap"); return PNE_EDEGENERATE; }
    for (size_t b = 0; b < B && !p->user_proj; ++b)
        if (p->bp_iters[b] == 0) {
            set_error(ctx, PNE_ENOCONV, "BP did not converge for tensor set " + std::to_string(b));
            return PNE_ENOCONV;
        }
    return PNE_OK;
}

pne_status partition_settle(pne_ctx *ctx, pne_partition *p)
{
    if (!p->rec_pending) return PNE_OK;
    const size_t bytes = (size_t)p->n_sets * 12 + 16;
    std::vector<char> rec(bytes);
    char *h = (char *)pinned_slot(0, bytes);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h ? h : rec.data(), p->rec_dev.ptr, bytes, cudaMemcpyDeviceToHost, p->last_stream));
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(p->last_stream));
    if (h) std::memcpy(rec.data(), h, bytes);
    return partition_record(ctx, p, rec.data());
}

// Reads the deferred records of several partitions: every copy queued on its
// partition's stream, then one wait per distinct stream.  Returns the first
// non-OK record status (all records are read either way).
pne_status partition_settle_many(pne_ctx *ctx, const std::vector<pne_partition *> &ps)
{
    std::vector<pne_partition *> pend;
    size_t total = 0;
    for (pne_partition *p : ps)
        if (p->rec_pending && std::find(pend.begin(), pend.end(), p) == pend.end()) {
            pend.push_back(p);
            total += ((size_t)p->n_sets * 12 + 16 + 15) & ~size_t(15);
        }
    if (pend.empty()) return PNE_OK;
    std::vector<char> fallback;
    char *h = (char *)pinned_slot(0, total);
    if (!h) { fallback.assign(total, 0); h = fallback.data(); }
    std::vector<cudaStream_t> streams;
    size_t off = 0;
    for (pne_partition *p : pend) {
        const size_t bytes = (size_t)p->n_sets * 12 + 16;
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h + off, p->rec_dev.ptr, bytes, cudaMemcpyDeviceToHost, p->last_stream));
        if (std::find(streams.begin(), streams.end(), p->last_stream) == streams.end()) streams.push_back(p->last_stream);
        off += (bytes + 15) & ~size_t(15);
    }
    for (cudaStream_t st : streams) PNE_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    pne_status first = PNE_OK;
    off = 0;
    for (pne_partition *p : pend) {
        const size_t bytes = (size_t)p->n_sets * 12 + 16;
        const pne_status st = partition_record(ctx, p, h + off);
        if (st != PNE_OK && first == PNE_OK) first = st;
        off += (bytes + 15) & ~size_t(15);
    }
    return first;
}

}  // namespace pne

using namespace pne;

extern "C" {

pne_status pne_ctx_create(int device, pne_ctx **out)
{
    if (!out) return PNE_EINVAL;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || device < 0 || device >= n) {
        g_last_error = std::string("no CUDA device ") + std::to_string(device) +
                       (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string());
        return PNE_ECUDA;
    }
    e = cudaSetDevice(device);
    if (e != cudaSuccess) { g_last_error = cudaGetErrorString(e); return PNE_ECUDA; }
    pne_ctx *c = new pne_ctx();
    c->device = device;
    e = cudaStreamCreateWithFlags(&c->release_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { g_last_error = cudaGetErrorString(e); delete c; return PNE_ECUDA; }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    // PNE_SEARCH_ARENA_MAX (nodes) lowers the node-arena limit of the cluster
    // search, so that the depth-first completion below the deepest level that
    // fits can be exercised on small networks
    if (const char *lim = std::getenv("PNE_SEARCH_ARENA_MAX")) c->arena_max = std::max(0LL, std::atoll(lim));
    // keep stream-ordered allocations pooled inside this process
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = std::numeric_limits<uint64_t>::max();
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    *out = c;
    return PNE_OK;
}

void pne_ctx_destroy(pne_ctx *ctx)
{
    if (!ctx) return;
    {
        // cached records and geometries are released on the release stream
        // after the streams that used them (which may be gone by now)
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        ctx->enum_cache.clear();
        ctx->geom_cache.clear();
    }
    cudaDeviceSynchronize();
    if (ctx->release_stream) cudaStreamDestroy(ctx->release_stream);
    for (auto ev : ctx->event_pool) cudaEventDestroy(ev);
    for (auto &pb : ctx->pinned_pool) cudaFreeHost(pb.first);
    if (ctx->side_ready) {
        for (auto st : ctx->side) cudaStreamDestroy(st);
        for (auto ev : ctx->side_ev) cudaEventDestroy(ev);
    }
    for (auto &l : ctx->stream_pool) {
        cudaStreamDestroy(l.s);
        cudaEventDestroy(l.fork);
        cudaEventDestroy(l.join);
    }
    delete ctx;
}

const char *pne_last_error(pne_ctx *ctx)
{
    (void)ctx;
    return g_last_error.c_str();
}

pne_status pne_ctx_set_allocator(pne_ctx *ctx, pne_alloc_fn alloc, pne_free_fn free_fn, void *user)
{
    if (!ctx || (!alloc) != (!free_fn)) return PNE_EINVAL;
    ctx->alloc = alloc; ctx->free_fn = free_fn; ctx->alloc_user = user;
    return PNE_OK;
}

pne_status pne_build_partition(pne_ctx *ctx, const pne_network *net, const pne_partition_opts *opts,
                               void *stream, pne_partition **out)
{
    HostScope hs__(ctx, "partition");
    if (!ctx || !out) return PNE_EINVAL;
    *out = nullptr;
    pne_status st;
    {
        HostScope hv__(ctx, "part_validate");
        if ((st = validate(ctx, net))) return st;
    }
    cudaStream_t s = (cudaStream_t)stream;
    double tol = (opts && opts->tol > 0) ? opts->tol : 1e-13;
    int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 10000;
    double damping = opts ? opts->damping : 0.0;
    if (!(damping >= 0.0 && damping < 1.0)) { set_error(ctx, PNE_EINVAL, "damping must be in [0,1)"); return PNE_EINVAL; }

    pne_partition *p = new pne_partition();
    p->ctx = ctx;
    p->last_stream = s;
    const int N = net->n_sites, M = net->n_bonds;
    if ((st = get_geometry(ctx, net, s, p->geo))) { delete p; return st; }
    const Geometry &f = p->geo->full, &c = p->geo->closed;
    int64_t slices = 1;
    for (int d : p->geo->open_dims) slices *= d;
    if (slices > 4096) { delete p; set_error(ctx, PNE_EINVAL, "more than 4096 open-index assignments"); return PNE_EINVAL; }
    p->n_sets = net->n_batch;
    p->n_slices = (int)slices;
    p->n_members = p->n_sets * p->n_slices;
    const int64_t fstride = f.tens_off[N], cstride = c.tens_off[N];
    const size_t B = p->n_sets, Bm = p->n_members;
    HostScope ha__(ctx, "part_alloc");
    {
        // one allocation, carved into the partition's buffers (256-byte aligned)
        DevBuf *parts[] = {&p->T, &p->msg, &p->gauge, &p->Mb, &p->site_info, &p->site_scale, &p->vac,
                           &p->rec_dev, &p->site_zero};
        const size_t sizes[] = {B * fstride * 8, 2 * B * f.n_legs * kMsgStride * 8, B * std::max(M, 1) * 2 * 64 * 8,
                                Bm * cstride * 8, Bm * N * 8, Bm * N * 8, Bm * 3 * 8,
                                (opts && opts->async_status) ? B * 12 + 16 : 0, Bm * N};
        size_t total = 0;
        for (size_t i = 0; i < sizeof sizes / sizeof sizes[0]; ++i) total += (sizes[i] + 255) & ~size_t(255);
        if ((st = dev_alloc(ctx, p->storage, total, s))) { pne_partition_destroy(p); return st; }
        char *at = (char *)p->storage.ptr;
        for (size_t i = 0; i < sizeof sizes / sizeof sizes[0]; ++i) {
            parts[i]->ptr = sizes[i] ? at : nullptr;
            parts[i]->bytes = sizes[i];
            at += (sizes[i] + 255) & ~size_t(255);
        }
    }
    // input tensors: a host or device source, in one copy
    {
        const size_t bytes = B * fstride * 8;
        cudaError_t e = cudaMemcpyAsync(p->T.ptr, net->data, bytes,
                                        net->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) { pne_partition_destroy(p); set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
    }
    ha__.stop();
    p->bp_iters.assign(B, 0);
    p->bp_residual.assign(B, 0.0);
    // convergence record: read back with the final synchronisation
    char *rb = (char *)pinned_slot(0, B * 12 + 16);
    std::vector<char> rb_fallback;
    if (!rb) { rb_fallback.assign(B * 12 + 16, 0); rb = rb_fallback.data(); }
    double *h_res = (double *)rb;
    int32_t *flags = (int32_t *)(rb + B * 8);
    int32_t *h_iters = flags + 4;
    std::memset(rb, 0, B * 12 + 16);
    const int arith = opts ? opts->arithmetic : 0;
    if (arith != 0 && arith != 1) { pne_partition_destroy(p); set_error(ctx, PNE_EINVAL, "arithmetic must be 0 or 1"); return PNE_EINVAL; }
    p->arithmetic = arith;
    const bool user = opts && opts->use_user_projectors;
    if (user && (!opts->user_u || !opts->user_v)) {
        pne_partition_destroy(p);
        set_error(ctx, PNE_EINVAL, "use_user_projectors needs user_u and user_v");
        return PNE_EINVAL;
    }
    p->user_proj = user;
    // the projectors: BP sweeps to a fixed point, or the caller's vectors
    auto projectors = [&](void *rec, cudaMemcpyKind kind) {
        return user ? launch_user_projectors(ctx, p, opts->user_u, opts->user_v, s, rec, kind)
                    : launch_bp(ctx, p, tol, max_iter, damping, s, rec, arith, kind);
    };
    if (opts && opts->async_status) {
        // deferred record: kept on the device, read by the next synchronising call
        char *rd = (char *)p->rec_dev.ptr;
        if ((st = projectors(rd, cudaMemcpyDeviceToDevice)) ||
            (st = launch_gauge(ctx, p, s, nullptr))) {
            pne_partition_destroy(p);
            return st ? st : PNE_ECUDA;
        }
        p->rec_pending = true;
        *out = p;
        return PNE_OK;
    }
    if ((st = projectors(rb, cudaMemcpyDeviceToHost)) || (st = launch_gauge(ctx, p, s, nullptr))) {
        pne_partition_destroy(p);
        return st;
    }
    cudaError_t e;
    {
        HostScope hw__(ctx, "sync_partition");
        e = cudaStreamSynchronize(s);
    }
    if (e != cudaSuccess) { pne_partition_destroy(p); set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
    std::memcpy(p->bp_iters.data(), h_iters, B * 4);
    std::memcpy(p->bp_residual.data(), h_res, B * 8);
    if (flags[0] || flags[2]) { pne_partition_destroy(p); set_error(ctx, PNE_ETIMEOUT, "grid barrier timed out in BP"); return PNE_ETIMEOUT; }
    if (flags[1] || flags[3]) { pne_partition_destroy(p); set_error(ctx, PNE_EDEGENERATE, "zero message or zero message overlap"); return PNE_EDEGENERATE; }
    *out = p;
    for (size_t b = 0; b < B && !p->user_proj; ++b)
        if (p->bp_iters[b] == 0) {
            set_error(ctx, PNE_ENOCONV, "BP did not converge for tensor set " + std::to_string(b));
            return PNE_ENOCONV;
        }
    return PNE_OK;
}

void pne_partition_destroy(pne_partition *p)
{
    if (!p) return;
    pne_ctx *ctx = p->ctx;
    // released after the partition's own stream and the streams of the terms
    // handles that read it (destroyed before it) reach their last use
    cudaStream_t s = ctx->release_stream;
    p->uses.note(ctx, p->last_stream);
    if (!p->uses.join(s)) { cudaDeviceSynchronize(); s = nullptr; }
    p->uses.release(ctx);
    // the partition's buffers are views of one allocation; the converted
    // copies are allocated on demand
    DevBuf *bufs[] = {&p->storage, &p->Mb32, &p->Mb16, &p->rec_own};
    for (DevBuf *b : bufs) dev_free(ctx, *b, s);
    if (p->geo) p->geo->uses.note(ctx, s);        // the geometry outlives every use of the partition
    delete p;
}

pne_status pne_enumerate_terms(pne_ctx *ctx, const pne_partition *part, const pne_enum_opts *opts,
                               void *stream, pne_terms **out, uint64_t *n_clusters, uint64_t *n_terms)
{
    HostScope hs__(ctx, "enumerate");
    if (!ctx || !part || !opts || !out) return PNE_EINVAL;
    *out = nullptr;
    const int K = opts->max_order, mode = opts->mode;
    if (K < 0 || K > kMaxOrder) { set_error(ctx, PNE_EINVAL, "max_order must be in 0..32"); return PNE_EINVAL; }
    if (mode != PNE_MODE_LOOP && mode != PNE_MODE_ALL) { set_error(ctx, PNE_EINVAL, "unknown mode"); return PNE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const Geometry &g = part->geo->closed;
    // the geometry tables may have been queued on the partition's stream
    if (part->geo->ready) PNE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, part->geo->ready, 0));
    // cluster-size cap (LOOP mode): clusters up to Kc bonds, terms up to K
    const int Kc = (mode == PNE_MODE_LOOP && opts->max_cluster > 0 && opts->max_cluster < K) ? opts->max_cluster : K;
    if (opts->max_cluster < 0) { set_error(ctx, PNE_EINVAL, "max_cluster must be >= 0"); return PNE_EINVAL; }
    std::string key = std::to_string(g.hash) + ":" + std::to_string(g.n_sites) + ":" + std::to_string(g.n_bonds) +
                      ":" + std::to_string(K) + ":" + std::to_string(mode) + ":" + std::to_string(Kc);
    std::shared_ptr<EnumRecord> rec;
    if (opts->use_cache) {
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        auto it = ctx->enum_cache.find(key);
        if (it != ctx->enum_cache.end()) rec = it->second;
    }
    pne_status st;
    if (!rec) {
        rec = std::make_shared<EnumRecord>();
        rec->ctx = ctx;
        // every exit, failures included, leaves the record's memory fenced
        // behind the work this call queued for it (on `s` and on the shape
        // stage's stream), so that it is never released under a running kernel
        struct Fence {
            pne_ctx *ctx; EnumRecord *r; cudaStream_t s; cudaStream_t sb = nullptr;
            ~Fence() { r->uses.note(ctx, s); if (sb && sb != s) r->uses.note(ctx, sb); }
        } fence{ctx, rec.get(), s};
        if (mode == PNE_MODE_ALL) {
            if (g.n_bonds > kMaxAllBonds || g.n_sites > 64) {
                set_error(ctx, PNE_EINVAL, "ALL mode needs <= 30 closed bonds and <= 64 sites"); return PNE_EINVAL;
            }
            rec->K = K; rec->mode = mode; rec->n_closed = g.n_bonds;
            rec->size_start.assign(K + 2, 0);
            rec->terms_by_order.assign(K + 1, 0);
            uint64_t tot = 0;
            for (int k = 0; k <= K && k <= g.n_bonds; ++k) {
                double bn = 1.0;
                for (int i = 1; i <= k; ++i) bn = bn * (g.n_bonds - k + i) / i;
                rec->terms_by_order[k] = (uint64_t)llround(bn);
                tot += rec->terms_by_order[k];
            }
            rec->n_terms = tot;
        } else {
            if (K == 0) {
                rec->K = 0; rec->mode = mode; rec->size_start.assign(2, 0);
                rec->terms_by_order.assign(1, 1); rec->n_terms = 1;
                rec->width = 1; rec->vwidth = 1;
            } else {
                {
                    HostScope h1(ctx, "enum_clusters");
                    if ((st = enumerate_clusters(ctx, g, Kc, mode, *rec, s))) return st;
                    if (Kc < K) {
                        // no cluster is larger than Kc: the size groups Kc+1..K are empty
                        rec->K = K;
                        rec->size_start.resize(K + 2, rec->size_start[Kc + 1]);
                    }
                }
                // the shape stage (contraction plans) and the term stage run on
                // two streams, their host waits interleaved: each waits for its
                // own readback while the other's work runs
                ShapePrep sp;
                TuplePrep tp;
                pne_ctx::Lent ls;
                const bool shapes = shapes_needed(g, *rec);
                cudaStream_t sb = s;
                if (shapes) {
                    std::lock_guard<std::mutex> lk(ctx->pool_mu);
                    if (!ctx->stream_pool.empty()) {
                        ls = ctx->stream_pool.back();
                        ctx->stream_pool.pop_back();
                    }
                }
                auto fail = [&](pne_status e) {
                    // buffers of the unfinished stages are released behind the
                    // kernels already queued on their streams
                    shapes_release(ctx, sp, sb);
                    tuples_abort(ctx, tp, s);
                    fence.sb = sb;
                    if (ls.s) { std::lock_guard<std::mutex> lk(ctx->pool_mu); ctx->stream_pool.push_back(ls); }
                    return e;
                };
                if (shapes) {
                    if (!ls.s) {
                        // the shape stage sits on the enumeration's critical path: the
                        // device's highest stream priority, so its small launches are
                        // scheduled ahead of other streams' waiting blocks
                        int least = 0, greatest = 0;
                        cudaDeviceGetStreamPriorityRange(&least, &greatest);
                        PNE_CUDA_TRY(ctx, cudaStreamCreateWithPriority(&ls.s, cudaStreamNonBlocking, greatest));
                        PNE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ls.fork, cudaEventDisableTiming));
                        PNE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ls.join, cudaEventDisableTiming));
                    }
                    sb = ls.s;
                    fence.sb = sb;
                    if (cudaEventRecord(ls.fork, s) != cudaSuccess || cudaStreamWaitEvent(sb, ls.fork, 0) != cudaSuccess)
                        return fail(PNE_ECUDA);
                }
                {
                    HostScope h2(ctx, "enum_shapes_begin");
                    if ((st = shapes_begin(ctx, g, *rec, sp, sb))) return fail(st);
                }
                {
                    HostScope h3(ctx, "enum_tuples_begin");
                    if ((st = tuples_begin(ctx, *rec, tp, s))) return fail(st);
                }
                {
                    HostScope h4(ctx, "enum_shapes_plan");
                    if ((st = shapes_plan(ctx, g, *rec, sp, sb))) return fail(st);
                }
                {
                    HostScope h5(ctx, "enum_tuples_finish");
                    if ((st = tuples_finish(ctx, *rec, tp, s))) return fail(st);
                }
                {
                    HostScope h6(ctx, "enum_shapes_complete");
                    if ((st = shapes_complete(ctx, g, *rec, sp, sb))) return fail(st);
                }
                if (ls.s) {
                    if (cudaEventRecord(ls.join, sb) != cudaSuccess || cudaStreamWaitEvent(s, ls.join, 0) != cudaSuccess)
                        return fail(PNE_ECUDA);
                    std::lock_guard<std::mutex> lk(ctx->pool_mu);
                    ctx->stream_pool.push_back(ls);
                }
                if ((st = sum_desc_prepare(ctx, *rec, s))) return st;
            }
        }
        if (opts->use_cache) {
            // a cached record may be used from other streams: finish it first
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
            std::lock_guard<std::mutex> lk(ctx->cache_mu);
            ctx->enum_cache[key] = rec;
        }
    }
    pne_terms *t = new pne_terms();
    t->ctx = ctx; t->part = part; t->rec = rec; t->K = K; t->mode = mode;
    t->last_stream = s;
    const size_t Bm = part->n_members;
    const size_t ncl = std::max<uint64_t>(rec->n_clusters, 1);
    if ((st = dev_alloc(ctx, t->status, 16, s))) { delete t; return st; }
    cudaMemsetAsync(t->status.ptr, 0, 16, s);
    if (mode == PNE_MODE_LOOP) {
        if ((st = dev_alloc(ctx, t->w, Bm * ncl * 8, s)) || (st = dev_alloc(ctx, t->nzc, Bm * ncl * 4, s))) {
            pne_terms_destroy(t); return st;
        }
    }
    // with the cache on, the handle's buffers are finished too (the server's
    // launcher uses them from its own stream); otherwise the lists and buffers
    // are ordered on `stream` like every other asynchronous call
    if (opts->use_cache) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { pne_terms_destroy(t); set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
    }
    *out = t;
    if (n_clusters) *n_clusters = rec->n_clusters;
    if (n_terms) *n_terms = rec->n_terms;
    return PNE_OK;
}

pne_status pne_enumerate_combinatorial(pne_ctx *ctx, const pne_partition *part, int32_t n_partitions,
                                       const int32_t *partition_ptr, const int32_t *partition_bonds, void *stream,
                                       pne_terms **out, uint64_t *n_components, uint64_t *n_terms)
{
    HostScope hs__(ctx, "enumerate_comb");
    if (!ctx || !part || !out || !partition_ptr || !partition_bonds) return PNE_EINVAL;
    *out = nullptr;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    const int M = n_partitions;
    if (M < 1 || M > 20) return bad("the combinatorial form takes 1..20 partitions");
    cudaStream_t s = (cudaStream_t)stream;
    const GeomPair &gp = *part->geo;
    const Geometry &g = gp.closed;
    const int N = g.n_sites, B = g.n_bonds;
    for (int b = 0; b < B; ++b)
        if (g.bond_dim[b] > kMaxDim - 1) return bad("the combinatorial form needs bond dimensions <= 7");
    // each partition as closed bond ids
    if (partition_ptr[0] != 0) return bad("partition_ptr[0] must be 0");
    std::vector<std::vector<int>> parts(M);
    for (int p = 0; p < M; ++p) {
        if (partition_ptr[p + 1] <= partition_ptr[p]) return bad("every partition needs at least one bond");
        for (int i = partition_ptr[p]; i < partition_ptr[p + 1]; ++i) {
            const int fb = partition_bonds[i];
            if (fb < 0 || fb >= gp.full.n_bonds) return bad("partition bond out of range");
            const int cb = gp.closed_of_full[fb];
            if (cb < 0) return bad("partitions transect closed bonds only");
            parts[p].push_back(cb);
        }
    }
    if (part->geo->ready) PNE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, part->geo->ready, 0));
    auto rec = std::make_shared<EnumRecord>();
    rec->ctx = ctx;
    rec->comb = true;
    rec->K = M;
    rec->mode = PNE_MODE_COMB;
    rec->n_closed = B;
    rec->empty_by_order.assign(M + 1, 0);
    struct Fence {
        pne_ctx *ctx; EnumRecord *r; cudaStream_t s;
        ~Fence() { r->uses.note(ctx, s); }
    } fence{ctx, rec.get(), s};
    // every sub-network: union-find over the sites along its kept bonds; the
    // distinct components become the record's clusters
    std::map<std::vector<int32_t>, int32_t> comp_id;
    std::vector<std::vector<int32_t>> comps;
    std::vector<std::vector<std::pair<int, std::vector<int32_t>>>> by_m;   // [m] -> (order, component ids)
    std::vector<int> parent(N), cut(B);
    std::function<int(int)> find = [&](int x) { while (parent[x] != x) { parent[x] = parent[parent[x]]; x = parent[x]; } return x; };
    for (uint32_t x = 1; x < (1u << M); ++x) {
        std::fill(cut.begin(), cut.end(), 0);
        int order = 0;
        for (int p = 0; p < M; ++p)
            if (x >> p & 1) { ++order; for (int b : parts[p]) cut[b] = 1; }
        for (int v = 0; v < N; ++v) parent[v] = v;
        for (int b = 0; b < B; ++b)
            if (!cut[b]) {
                const int a = find(g.bond_site[2 * b]), c = find(g.bond_site[2 * b + 1]);
                if (a != c) parent[a] = c;
            }
        std::map<int, std::vector<int32_t>> groups;          // root -> kept bonds (ascending)
        for (int b = 0; b < B; ++b)
            if (!cut[b]) groups[find(g.bond_site[2 * b])].push_back(b);
        if (groups.empty()) { rec->empty_by_order[order] += 1; continue; }
        std::vector<int32_t> ids;
        for (auto &kv : groups) {
            if (kv.second.size() > (size_t)kMaxOrder) return bad("a component of a sub-network has more than 32 bonds");
            auto it = comp_id.find(kv.second);
            int32_t id;
            if (it == comp_id.end()) {
                id = (int32_t)comps.size();
                comp_id.emplace(kv.second, id);
                comps.push_back(kv.second);
            } else {
                id = it->second;
            }
            ids.push_back(id);
        }
        std::sort(ids.begin(), ids.end());
        const size_t m = ids.size();
        if (by_m.size() < m + 1) by_m.resize(m + 1);
        by_m[m].push_back({order, ids});
    }
    const int64_t nc = (int64_t)comps.size();
    int width = 1, vwidth = 1;
    std::vector<std::vector<int32_t>> verts(nc);
    for (int64_t c = 0; c < nc; ++c) {
        std::vector<int32_t> vs;
        for (int b : comps[c]) { vs.push_back(g.bond_site[2 * b]); vs.push_back(g.bond_site[2 * b + 1]); }
        std::sort(vs.begin(), vs.end());
        vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
        if (vs.size() > 32) return bad("a component of a sub-network has more than 32 sites");
        verts[c] = vs;
        width = std::max(width, (int)comps[c].size());
        vwidth = std::max(vwidth, (int)vs.size());
    }
    rec->width = width;
    rec->vwidth = vwidth;
    rec->n_clusters = (uint64_t)nc;
    rec->size_start.assign(M + 2, 0);                     // no single-cluster terms: every term is a level entry
    if (by_m.size() > 17) {
        set_error(ctx, PNE_EOVERFLOW, "a sub-network has more than 16 components");
        return PNE_EOVERFLOW;
    }
    pne_status st;
    {
        const size_t nn = std::max<int64_t>(nc, 1);
        std::vector<int32_t> he(nn * width, -1), hv(nn * vwidth, -1), hs(nn, 0);
        for (int64_t c = 0; c < nc; ++c) {
            for (size_t j = 0; j < comps[c].size(); ++j) he[c * width + j] = comps[c][j];
            for (size_t j = 0; j < verts[c].size(); ++j) hv[c * vwidth + j] = verts[c][j];
            hs[c] = (int32_t)comps[c].size();
        }
        if ((st = dev_alloc(ctx, rec->cl_edges, he.size() * 4, s)) || (st = dev_alloc(ctx, rec->cl_verts, hv.size() * 4, s)) ||
            (st = dev_alloc(ctx, rec->cl_size, hs.size() * 4, s)) ||
            (st = upload(ctx, rec->cl_edges.ptr, he.data(), he.size() * 4, s)) ||
            (st = upload(ctx, rec->cl_verts.ptr, hv.data(), hv.size() * 4, s)) ||
            (st = upload(ctx, rec->cl_size.ptr, hs.data(), hs.size() * 4, s)))
            return st;
    }
    // the terms, one level per number of components, ordered by |x|
    rec->terms_by_order.assign(M + 1, 0);
    rec->n_terms = 0;
    for (int k = 1; k <= M; ++k) rec->terms_by_order[k] += rec->empty_by_order[k];
    for (size_t m = 1; m < by_m.size(); ++m) {
        auto &lst = by_m[m];
        if (lst.empty()) continue;
        std::stable_sort(lst.begin(), lst.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
        EnumRecord::Level L;
        L.m = (int)m;
        L.n = lst.size();
        L.order_start.assign(M + 2, 0);
        std::vector<int32_t> idx(lst.size() * m);
        for (size_t i = 0; i < lst.size(); ++i) {
            for (size_t j = 0; j < m; ++j) idx[i * m + j] = lst[i].second[j];
            rec->terms_by_order[lst[i].first] += 1;
        }
        for (int k = 0; k <= M + 1; ++k) {
            int64_t n = 0;
            for (auto &e : lst) n += (e.first < k);
            L.order_start[k] = n;
        }
        if ((st = dev_alloc(ctx, L.idx, idx.size() * 4, s)) || (st = upload(ctx, L.idx.ptr, idx.data(), idx.size() * 4, s)))
            return st;
        rec->levels.push_back(L);
    }
    for (int k = 0; k <= M; ++k) rec->n_terms += rec->terms_by_order[k];
    // the virtual geometry (bond dimensions d + 1) and the contraction plans
    Geometry &vg = rec->vgeo;
    vg.n_sites = N; vg.n_bonds = B;
    vg.bond_site = g.bond_site; vg.site_ptr = g.site_ptr; vg.site_bonds = g.site_bonds;
    vg.bond_dim = g.bond_dim;
    for (auto &d : vg.bond_dim) d += 1;
    if ((st = finish_geometry(ctx, vg, s))) return st;
    if (nc > 0) {
        ShapePrep sp;
        if ((st = shapes_begin(ctx, vg, *rec, sp, s)) || (st = shapes_plan(ctx, vg, *rec, sp, s)) ||
            (st = shapes_complete(ctx, vg, *rec, sp, s))) {
            shapes_release(ctx, sp, s);
            return st;
        }
    }
    pne_terms *t = new pne_terms();
    t->ctx = ctx; t->part = part; t->rec = rec; t->K = M; t->mode = PNE_MODE_COMB;
    t->last_stream = s;
    const size_t Bm = part->n_members;
    const size_t ncl = std::max<int64_t>(nc, 1);
    if ((st = dev_alloc(ctx, t->status, 16, s)) || (st = dev_alloc(ctx, t->w, Bm * ncl * 8, s)) ||
        (st = dev_alloc(ctx, t->nzc, Bm * ncl * 4, s))) {
        pne_terms_destroy(t);
        return st;
    }
    cudaMemsetAsync(t->status.ptr, 0, 16, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { pne_terms_destroy(t); set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
    *out = t;
    if (n_components) *n_components = (uint64_t)nc;
    if (n_terms) *n_terms = rec->n_terms;
    return PNE_OK;
}

void pne_terms_destroy(pne_terms *t)
{
    if (!t) return;
    cudaStream_t s = t->last_stream;
    if (t->rec) t->rec->uses.note(t->ctx, s);    // the record outlives this stream's queued work
    // so does the partition (terms handles are destroyed before it)
    if (t->part) const_cast<pne_partition *>(t->part)->uses.note(t->ctx, s);
    dev_free(t->ctx, t->Mf, s);
    dev_free(t->ctx, t->Mf32, s);
    dev_free(t->ctx, t->Mf16, s);
    dev_free(t->ctx, t->w, s);
    dev_free(t->ctx, t->nzc, s);
    dev_free(t->ctx, t->sums, s);
    dev_free(t->ctx, t->status, s);
    dev_free(t->ctx, t->sum_done, s);
    delete t;
}

pne_status pne_contract_terms(pne_ctx *ctx, pne_terms *t, pne_dtype dtype, void *stream)
{
    HostScope hs__(ctx, "contract");
    if (!ctx || !t) return PNE_EINVAL;
    if (dtype < PNE_F64 || dtype > PNE_BF16) { set_error(ctx, PNE_EINVAL, "unknown dtype"); return PNE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    t->last_stream = s;
    pne_status st = (t->mode == PNE_MODE_ALL) ? launch_all_mode(ctx, t, dtype, s) : launch_contract(ctx, t, dtype, s);
    if (st) return st;
    t->dtype = dtype;
    t->contracted = true;
    return PNE_OK;
}

int64_t pne_terms_n_results(const pne_terms *t)
{
    return t && t->part ? (int64_t)t->part->n_members : 0;
}

pne_status pne_open_tensor_assemble(const pne_result *res, int64_t n_sets, int64_t n_open, double *out,
                                    double *log_scale)
{
    if (!res || !out || !log_scale || n_sets < 1 || n_open < 1) return PNE_EINVAL;
    for (int64_t b = 0; b < n_sets; ++b) {
        const pne_result *r = res + b * n_open;
        double m = -std::numeric_limits<double>::infinity();
        for (int64_t o = 0; o < n_open; ++o)
            if (r[o].sign != 0 && std::isfinite(r[o].log_abs)) m = std::max(m, r[o].log_abs);
        log_scale[b] = m;
        for (int64_t o = 0; o < n_open; ++o) {
            const bool zero = r[o].sign == 0 || !std::isfinite(r[o].log_abs) || !std::isfinite(m);
            out[b * n_open + o] = zero ? 0.0 : r[o].sign * std::exp(r[o].log_abs - m);
        }
    }
    return PNE_OK;
}

pne_status pne_open_tensor(pne_ctx *ctx, const pne_terms *t, void *stream, double *out, double *log_scale)
{
    if (!ctx || !t || !out || !log_scale) return PNE_EINVAL;
    const pne_partition *p = t->part;
    std::vector<pne_result> res((size_t)p->n_members);
    const pne_status st = pne_sum(ctx, t, stream, res.data());
    if (st != PNE_OK && st != PNE_ENOCONV) return st;
    const pne_status sa = pne_open_tensor_assemble(res.data(), p->n_sets, p->n_slices, out, log_scale);
    return sa != PNE_OK ? sa : st;
}

pne_status pne_terms_export(pne_ctx *ctx, const pne_terms *t, void *stream, int32_t *edges, double *w)
{
    if (!ctx || !t) return PNE_EINVAL;
    if (t->mode != PNE_MODE_LOOP && t->mode != PNE_MODE_COMB) {
        set_error(ctx, PNE_EINVAL, "export needs LOOP or COMB mode");
        return PNE_EINVAL;
    }
    const int row = (t->mode == PNE_MODE_COMB) ? kMaxOrder : t->K;    // entries per exported cluster row
    cudaStream_t s = (cudaStream_t)stream;
    const_cast<pne_terms *>(t)->last_stream = s;
    const EnumRecord &rec = *t->rec;
    const size_t n = rec.n_clusters;
    if (n == 0) return PNE_OK;
    if (edges) {
        std::vector<int32_t> buf(n * rec.width);
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(buf.data(), rec.cl_edges.ptr, buf.size() * 4, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        std::vector<int32_t> full_of_closed;
        for (size_t b = 0; b < t->part->geo->closed_of_full.size(); ++b)
            if (t->part->geo->closed_of_full[b] >= 0) full_of_closed.push_back((int32_t)b);
        for (size_t i = 0; i < n; ++i)
            for (int j = 0; j < row; ++j) {
                const int32_t e = (j < rec.width) ? buf[i * rec.width + j] : -1;
                edges[i * row + j] = (e >= 0) ? full_of_closed[e] : -1;
            }
    }
    if (w) {
        if (!t->contracted) { set_error(ctx, PNE_EINVAL, "contract before exporting values"); return PNE_EINVAL; }
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(w, t->w.ptr, n * t->part->n_members * 8, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    return PNE_OK;
}

pne_status pne_sum(pne_ctx *ctx, const pne_terms *t, void *stream, pne_result *out)
{
    HostScope hs__(ctx, "sum");
    if (!ctx || !t || !out) return PNE_EINVAL;
    if (!t->contracted) { set_error(ctx, PNE_EINVAL, "pne_contract_terms must run before pne_sum"); return PNE_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const_cast<pne_terms *>(t)->last_stream = s;
    const pne_partition *p = t->part;
    const int K = t->K, B = p->n_members;
    std::vector<double> c, a;
    int32_t status = 0;
    // the vacuum record (and a deferred BP record) are read back with the sums:
    // one synchronisation
    const size_t vbytes = (size_t)B * 3 * 8;
    const size_t rbytes = p->rec_pending ? (size_t)p->n_sets * 12 + 16 : 0;
    std::vector<char> hb(vbytes + rbytes);
    char *hp = (char *)pinned_slot(2, vbytes + rbytes);
    char *dst = hp ? hp : hb.data();
    std::vector<D2HCopy> extra{{dst, p->vac.ptr, vbytes}};
    if (rbytes) extra.push_back({dst + vbytes, p->rec_dev.ptr, rbytes});
    pne_status st = launch_sums(ctx, t, s, c, a, &status, extra);
    if (st) return st;
    if (hp) std::memcpy(hb.data(), hp, vbytes + rbytes);
    const double *vac = (const double *)hb.data();
    pne_status bp_st = PNE_OK;
    if (rbytes) bp_st = partition_record(ctx, const_cast<pne_partition *>(p), hb.data() + vbytes);
    if (status) { set_error(ctx, PNE_EOVERFLOW, "a cluster exceeded the contraction buffer"); return PNE_EOVERFLOW; }
    for (int b = 0; b < B; ++b) {
        const int set = b / p->n_slices;
        if (t->rec->comb) {
            // sub-networks with no kept bond are the capped sites alone: 1
            // relative to Z_ref, unless a capped site is zero
            double *cb = &c[(size_t)b * (K + 1)], *ab = &a[(size_t)b * (K + 1)];
            if ((int)vac[3 * (size_t)b + 2] == 0)
                for (int k = 0; k <= K; ++k) { cb[k] += (double)t->rec->empty_by_order[k]; ab[k] += (double)t->rec->empty_by_order[k]; }
            finalize_comb_result(out[b], K, t->dtype, cb, ab, &vac[3 * (size_t)b], t->rec->n_terms, t->rec->n_clusters,
                                 p->geo->closed.n_sites, p->bp_iters[set], p->bp_residual[set]);
            continue;
        }
        finalize_result(out[b], K, t->mode, t->dtype, &c[(size_t)b * (K + 1)], &a[(size_t)b * (K + 1)], &vac[3 * (size_t)b],
                        t->rec->n_terms, t->rec->n_clusters, p->bp_iters[set], p->bp_residual[set]);
    }
    return bp_st;
}

pne_status pne_partition_update(pne_ctx *ctx, pne_partition *p, const double *data, int32_t data_on_device,
                                const pne_partition_opts *opts, void *stream)
{
    if (!ctx || !p || !data) return PNE_EINVAL;
    partition_settle(ctx, p);                 // a deferred record of the previous build is superseded
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    const double tol = (opts && opts->tol > 0) ? opts->tol : 1e-13;
    const int max_iter = (opts && opts->max_iter > 0) ? opts->max_iter : 10000;
    const double damping = opts ? opts->damping : 0.0;
    if (!(damping >= 0.0 && damping < 1.0)) { set_error(ctx, PNE_EINVAL, "damping must be in [0,1)"); return PNE_EINVAL; }
    const size_t bytes = (size_t)p->n_sets * p->geo->full.tens_off[p->geo->full.n_sites] * 8;
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(p->T.ptr, data, bytes, data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    const size_t B = p->n_sets;
    char *rb = (char *)pinned_slot(0, B * 12 + 16);
    std::vector<char> rb_fallback;
    if (!rb) { rb_fallback.assign(B * 12 + 16, 0); rb = rb_fallback.data(); }
    double *h_res = (double *)rb;
    int32_t *flags = (int32_t *)(rb + B * 8);
    int32_t *h_iters = flags + 4;
    std::memset(rb, 0, B * 12 + 16);
    pne_status st;
    const int arith = opts ? opts->arithmetic : p->arithmetic;
    if (arith != 0 && arith != 1) { set_error(ctx, PNE_EINVAL, "arithmetic must be 0 or 1"); return PNE_EINVAL; }
    p->arithmetic = arith;
    const bool user = opts && opts->use_user_projectors;
    if (user && (!opts->user_u || !opts->user_v)) {
        set_error(ctx, PNE_EINVAL, "use_user_projectors needs user_u and user_v");
        return PNE_EINVAL;
    }
    p->user_proj = user;
    auto projectors = [&](void *rec, cudaMemcpyKind kind) {
        return user ? launch_user_projectors(ctx, p, opts->user_u, opts->user_v, s, rec, kind)
                    : launch_bp(ctx, p, tol, max_iter, damping, s, rec, arith, kind);
    };
    if (opts && opts->async_status) {
        // deferred record, read by the next call that synchronises
        if (!p->rec_dev.ptr) {
            if ((st = dev_alloc(ctx, p->rec_own, B * 12 + 16, s))) return st;
            p->rec_dev.ptr = p->rec_own.ptr;
            p->rec_dev.bytes = p->rec_own.bytes;
        }
        if ((st = projectors(p->rec_dev.ptr, cudaMemcpyDeviceToDevice)) || (st = launch_gauge(ctx, p, s, nullptr)))
            return st;
        p->mb32_dtype = -1;
        p->rec_pending = true;
        return PNE_OK;
    }
    if ((st = projectors(rb, cudaMemcpyDeviceToHost)) || (st = launch_gauge(ctx, p, s, nullptr)))
        return st;
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    std::memcpy(p->bp_iters.data(), h_iters, B * 4);
    std::memcpy(p->bp_residual.data(), h_res, B * 8);
    p->mb32_dtype = -1;
    if (flags[0] || flags[2]) { set_error(ctx, PNE_ETIMEOUT, "grid barrier timed out in BP"); return PNE_ETIMEOUT; }
    if (flags[1] || flags[3]) { set_error(ctx, PNE_EDEGENERATE, "zero message or zero message overlap"); return PNE_EDEGENERATE; }
    for (int b = 0; b < p->n_sets && !p->user_proj; ++b)
        if (p->bp_iters[b] == 0) { set_error(ctx, PNE_ENOCONV, "BP did not converge for tensor set " + std::to_string(b)); return PNE_ENOCONV; }
    return PNE_OK;
}

namespace {

double host_ms_now()
{
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Waits for the pending event pairs and folds them into the sums (and, when
// tracing, into the timeline).  Caller holds prof.mu.
void prof_drain(pne_ctx *ctx)
{
    auto &P = ctx->prof;
    for (auto &r : P.pending) {
        cudaEventSynchronize(r.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        auto &e = P.acc[r.name];
        e.first += 1;
        e.second += ms;
        if (P.trace && P.base && P.gpu_trace.size() < kTraceMax) {
            float t0 = 0.f;
            cudaEventElapsedTime(&t0, P.base, r.a);
            P.gpu_trace.push_back({r.name, r.s, (double)t0, (double)t0 + ms});
        }
        P.pool.push_back(r.a);
        P.pool.push_back(r.b);
    }
    P.pending.clear();
}

}  // namespace

pne_status pne_ctx_profile(pne_ctx *ctx, int enable)
{
    if (!ctx) return PNE_EINVAL;
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    auto &P = ctx->prof;
    for (auto &r : P.pending) { cudaEventSynchronize(r.b); P.pool.push_back(r.a); P.pool.push_back(r.b); }
    P.pending.clear();
    P.acc.clear();
    P.gpu_trace.clear();
    P.host_trace.clear();
    P.on = enable != 0;
    P.trace = enable == 2;
    if (P.trace) {
        // the origin: a device-wide idle point, then an event and the host
        // clock read as soon as that event has completed
        if (!P.base) PNE_CUDA_TRY(ctx, cudaEventCreate(&P.base));
        PNE_CUDA_TRY(ctx, cudaDeviceSynchronize());
        PNE_CUDA_TRY(ctx, cudaEventRecord(P.base, 0));
        PNE_CUDA_TRY(ctx, cudaEventSynchronize(P.base));
        P.host_base = host_ms_now();
    }
    return PNE_OK;
}

int pne_ctx_profile_read(pne_ctx *ctx, pne_profile_entry *out, int max)
{
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    prof_drain(ctx);
    std::vector<std::pair<std::string, std::pair<int64_t, double>>> v(ctx->prof.acc.begin(), ctx->prof.acc.end());
    std::sort(v.begin(), v.end(), [](const auto &x, const auto &y) { return x.second.second > y.second.second; });
    const int n = (int)v.size();
    for (int i = 0; i < n && i < max && out; ++i) {
        std::memset(out[i].name, 0, sizeof out[i].name);
        std::strncpy(out[i].name, v[i].first.c_str(), sizeof out[i].name - 1);
        out[i].launches = v[i].second.first;
        out[i].total_ms = v[i].second.second;
    }
    return n;
}

int pne_ctx_trace_read(pne_ctx *ctx, pne_trace_entry *out, int max, double *host_origin_ms)
{
    if (!ctx) return 0;
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    auto &P = ctx->prof;
    prof_drain(ctx);
    if (host_origin_ms) *host_origin_ms = P.host_base;
    // streams numbered in order of first appearance
    std::vector<cudaStream_t> ids;
    auto sid = [&](cudaStream_t st) {
        for (size_t i = 0; i < ids.size(); ++i)
            if (ids[i] == st) return (int)i;
        ids.push_back(st);
        return (int)ids.size() - 1;
    };
    std::vector<pne_trace_entry> v;
    v.reserve(P.gpu_trace.size() + P.host_trace.size());
    for (auto &r : P.gpu_trace) {
        pne_trace_entry e{};
        std::strncpy(e.name, r.name, sizeof e.name - 1);
        e.kind = 0;
        e.stream = sid(r.s);
        e.t0_ms = r.t0;
        e.t1_ms = r.t1;
        v.push_back(e);
    }
    for (auto &r : P.host_trace) {
        pne_trace_entry e{};
        std::strncpy(e.name, r.name, sizeof e.name - 1);
        e.kind = 1;
        e.stream = -1;
        e.t0_ms = r.t0;
        e.t1_ms = r.t1;
        v.push_back(e);
    }
    std::stable_sort(v.begin(), v.end(), [](const pne_trace_entry &x, const pne_trace_entry &y) { return x.t0_ms < y.t0_ms; });
    const int n = (int)v.size();
    for (int i = 0; i < n && i < max && out; ++i) out[i] = v[i];
    return n;
}

pne_status pne_terms_work(pne_ctx *ctx, const pne_terms *t, void *stream, uint64_t *fma_per_set)
{
    if (!ctx || !t || !fma_per_set) return PNE_EINVAL;
    if (t->mode != PNE_MODE_LOOP && t->mode != PNE_MODE_COMB) {
        set_error(ctx, PNE_EINVAL, "work count needs LOOP or COMB mode");
        return PNE_EINVAL;
    }
    if (t->rec->shaped) {
        uint64_t f = 0;
        for (int i = 0; i < t->rec->n_shapes; ++i) f += t->rec->shape_fma[i] * (uint64_t)t->rec->shape_count[i];
        *fma_per_set = f;
        return PNE_OK;
    }
    return launch_plan_work(ctx, t, (cudaStream_t)stream, fma_per_set);
}

pne_status pne_measure_fma_peak(pne_ctx *ctx, pne_dtype dtype, void *stream, double *flops_per_s)
{
    if (!ctx || !flops_per_s || (dtype != PNE_F64 && dtype != PNE_F32)) return PNE_EINVAL;
    return launch_fma_peak(ctx, dtype, (cudaStream_t)stream, flops_per_s);
}

}  // extern "C"

struct pne_batch {
    pne_ctx *ctx = nullptr;
    pne::BatchPlan *plan = nullptr;
    std::vector<pne_terms *> terms;
    int dtype = 0, wpb = 4, bps = 1, sched = PNE_SCHED_HANDLE;
    double tuned_ms = 0.0;
    bool use_graph = false;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t n_results = 0;
    cudaStream_t last = nullptr;          // stream of the last call that queued work for the batch
};

namespace {

// Launch shapes and work orders found by the autotuner, by batch signature
// (process-wide; g_tune_mu guards the map, its file and the one-time load).
struct TuneEntry {
    int wpb, bps, sched;
    double ms;
};
std::map<std::string, TuneEntry> g_tune_cache;
std::mutex g_tune_mu;
bool g_tune_loaded = false;

// file lines: "<key> <warps per block> <blocks per SM> <schedule> <ms>";
// lines of any other form are skipped
void tune_cache_load()
{
    const char *path = std::getenv("PNE_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char line[1024], key[512];
    int w, b, sc;
    double ms;
    while (std::fgets(line, sizeof(line), f))
        if (std::sscanf(line, "%511s %d %d %d %lf", key, &w, &b, &sc, &ms) == 5) g_tune_cache[key] = {w, b, sc, ms};
    std::fclose(f);
}

void tune_cache_store(const std::string &key, const TuneEntry &e)
{
    g_tune_cache[key] = e;
    const char *path = std::getenv("PNE_AUTOTUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d %d %.6f\n", key.c_str(), e.wpb, e.bps, e.sched, e.ms);
    std::fclose(f);
}

}  // namespace

extern "C" {

pne_status pne_batch_create(pne_ctx *ctx, int32_t n, pne_terms *const *terms, pne_dtype dtype,
                            const pne_batch_opts *opts, void *stream, pne_batch **out)
{
    if (!ctx || n < 1 || !terms || !out) return PNE_EINVAL;
    if (dtype < PNE_F64 || dtype > PNE_BF16) { set_error(ctx, PNE_EINVAL, "unknown dtype"); return PNE_EINVAL; }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    pne_batch *b = new pne_batch();
    b->ctx = ctx;
    b->dtype = dtype;
    b->last = s;
    b->terms.assign(terms, terms + n);
    for (pne_terms *t : b->terms) {
        if (!t) { delete b; return PNE_EINVAL; }
        t->last_stream = s;                       // conversions and tuning runs use the handles on `s`
        b->n_results += t->part->n_members;
        // the batch reports the BP record: read deferred ones now
        partition_settle(ctx, const_cast<pne_partition *>(t->part));
    }
    pne_status st = batch_plan_create(ctx, b->terms, dtype, s, &b->plan);
    if (st) { delete b; return st; }
    // launch shape: given, cached, or tuned by timing every candidate
    int w0 = opts ? opts->warps_per_block : 0, b0 = opts ? opts->blocks_per_sm : 0;
    const bool prof = ctx->prof.on;
    ctx->prof.on = false;
    if (w0 > 0 && b0 > 0) {
        const int sc = opts->schedule;
        if (sc != PNE_SCHED_HANDLE && sc != PNE_SCHED_LARGEST_FIRST) {
            ctx->prof.on = prof;
            pne_batch_destroy(b);
            set_error(ctx, PNE_EINVAL, "unknown batch schedule");
            return PNE_EINVAL;
        }
        if (w0 > 32 || batch_max_blocks_per_sm(b->plan, w0) < b0) {
            ctx->prof.on = prof;
            pne_batch_destroy(b);
            set_error(ctx, PNE_EINVAL, "launch shape does not fit (shared memory or occupancy)");
            return PNE_EINVAL;
        }
        b->wpb = w0; b->bps = b0; b->sched = sc;
    } else {
        std::unique_lock<std::mutex> tlk(g_tune_mu);
        if (!g_tune_loaded) { tune_cache_load(); g_tune_loaded = true; }
        uint64_t ncl = 0, nmem = 0;
        for (pne_terms *t : b->terms) { ncl += t->rec->n_clusters; nmem += t->part->n_members; }
        const std::string key = "v2_d" + std::to_string(dtype) + "_g" + std::to_string(n) + "_c" +
                                std::to_string(ncl) + "_m" + std::to_string(nmem) + "_sm" + std::to_string(ctx->n_sm);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            b->wpb = it->second.wpb; b->bps = it->second.bps; b->sched = it->second.sched; b->tuned_ms = it->second.ms;
        } else {
            // every (warps per block, blocks per SM, work order) that fits,
            // each run three times, the best of the last two kept
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0); cudaEventCreate(&e1);
            double best = 1e300;
            const int wcand[4] = {1, 2, 4, 8}, bcand[4] = {1, 2, 4, 8};
            const int scand[2] = {PNE_SCHED_HANDLE, PNE_SCHED_LARGEST_FIRST};
            for (int wi = 0; wi < 4; ++wi) {
                const int maxb = batch_max_blocks_per_sm(b->plan, wcand[wi]);
                for (int bi = 0; bi < 4; ++bi) {
                    if (bcand[bi] > maxb) continue;
                    if ((st = batch_prepare(ctx, b->plan, wcand[wi], bcand[bi], s))) {
                        ctx->prof.on = prof; pne_batch_destroy(b); return st;
                    }
                    for (int sc : scand) {
                        double t_best = 1e300;
                        for (int rep = 0; rep < 3; ++rep) {
                            cudaEventRecord(e0, s);
                            st = batch_enqueue(ctx, b->plan, wcand[wi], bcand[bi], sc, s);
                            cudaEventRecord(e1, s);
                            if (st || cudaEventSynchronize(e1) != cudaSuccess) {
                                ctx->prof.on = prof; pne_batch_destroy(b); return st ? st : PNE_ECUDA;
                            }
                            float ms = 0.f;
                            cudaEventElapsedTime(&ms, e0, e1);
                            if (rep > 0 && ms < t_best) t_best = ms;
                        }
                        if (t_best < best) { best = t_best; b->wpb = wcand[wi]; b->bps = bcand[bi]; b->sched = sc; }
                    }
                }
            }
            cudaEventDestroy(e0); cudaEventDestroy(e1);
            if (best >= 1e300) { ctx->prof.on = prof; pne_batch_destroy(b); set_error(ctx, PNE_EINVAL, "no launch shape fits"); return PNE_EINVAL; }
            b->tuned_ms = best;
            tune_cache_store(key, {b->wpb, b->bps, b->sched, best});
        }
    }
    if ((st = batch_prepare(ctx, b->plan, b->wpb, b->bps, s))) { ctx->prof.on = prof; pne_batch_destroy(b); return st; }
    b->use_graph = !opts || opts->use_graph;
    if (b->use_graph) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) { ctx->prof.on = prof; pne_batch_destroy(b); set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
        st = batch_enqueue(ctx, b->plan, b->wpb, b->bps, b->sched, b->cap);
        e = cudaStreamEndCapture(b->cap, &b->graph);
        if (st || e != cudaSuccess) { ctx->prof.on = prof; pne_batch_destroy(b); if (!st) set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return st ? st : PNE_ECUDA; }
        e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) { ctx->prof.on = prof; pne_batch_destroy(b); set_error(ctx, PNE_ECUDA, cudaGetErrorString(e)); return PNE_ECUDA; }
    }
    ctx->prof.on = prof;
    *out = b;
    return PNE_OK;
}

pne_status pne_batch_run(pne_ctx *ctx, pne_batch *b, void *stream, pne_result *out)
{
    if (!ctx || !b || !out) return PNE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    for (pne_terms *t : b->terms) t->last_stream = s;     // the handles' buffers are used on `s`
    if (b->use_graph) {
        ProfScope ps(ctx, s, "batch_graph");
        PNE_CUDA_TRY(ctx, cudaGraphLaunch(b->exec, s));
    } else {
        pne_status st = batch_enqueue(ctx, b->plan, b->wpb, b->bps, b->sched, s);
        if (st) return st;
    }
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (batch_status_host(b->plan)) { set_error(ctx, PNE_ETIMEOUT, "a batched sum waited too long"); return PNE_ETIMEOUT; }
    // convergence records deferred by asynchronous partition updates
    std::vector<pne_partition *> parts;
    for (const pne_terms *t : b->terms) parts.push_back(const_cast<pne_partition *>(t->part));
    const pne_status rec_st = partition_settle_many(ctx, parts);
    const double *h = batch_host_out(b->plan);
    const std::vector<int64_t> &off = batch_out_offsets(b->plan);
    int64_t r = 0;
    for (size_t g = 0; g < b->terms.size(); ++g) {
        const pne_terms *t = b->terms[g];
        const pne_partition *p = t->part;
        const int K = t->K;
        for (int m = 0; m < p->n_members; ++m) {
            const double *row = h + off[g] + (int64_t)m * ((K + 1) * 2 + 3);
            double c[kMaxOrder + 1], a[kMaxOrder + 1];
            for (int k = 0; k <= K; ++k) { c[k] = row[2 * k]; a[k] = row[2 * k + 1]; }
            const int set = m / p->n_slices;
            finalize_result(out[r++], K, t->mode, b->dtype, c, a, row + (K + 1) * 2, t->rec->n_terms, t->rec->n_clusters,
                            p->bp_iters[set], p->bp_residual[set]);
        }
    }
    return rec_st;
}

int64_t pne_batch_n_results(const pne_batch *b) { return b ? b->n_results : 0; }

pne_status pne_batch_config(const pne_batch *b, int32_t *warps_per_block, int32_t *blocks_per_sm, double *tuned_ms)
{
    if (!b) return PNE_EINVAL;
    if (warps_per_block) *warps_per_block = b->wpb;
    if (blocks_per_sm) *blocks_per_sm = b->bps;
    if (tuned_ms) *tuned_ms = b->tuned_ms;
    return PNE_OK;
}

pne_status pne_batch_schedule(const pne_batch *b, int32_t *schedule)
{
    if (!b || !schedule) return PNE_EINVAL;
    *schedule = b->sched;
    return PNE_OK;
}

void pne_batch_destroy(pne_batch *b)
{
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->plan) batch_plan_destroy(b->ctx, b->plan, b->last);
    delete b;
}

}  // extern "C"
