// Internal declarations shared by the translation units of libpne.
// Not part of the public ABI (include/pne.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>
#include <memory>
#include <atomic>
#include <map>
#include <mutex>

#include "pne.h"

namespace pne {

constexpr int kMaxDeg = PNE_MAX_DEG;
constexpr int kMaxDim = PNE_MAX_DIM;
constexpr int kMaxOrder = PNE_MAX_ORDER;
constexpr int kMsgStride = 8;            // doubles per stored message (>= kMaxDim)
constexpr int kBlkStride = 64;           // 2^kMaxDeg excitation masks per site
constexpr int kMaxAllBonds = 30;         // ALL mode: bitmask terms
constexpr int kWarpTensorMax = 1024;     // entries of one intermediate tensor per warp

// ------------------------------------------------------------------ index arithmetic
// q = r / d and m = r % d for 0 <= r < 2^22 - 1 and any d >= 1, without an
// integer divide: (r + 1/2) / d lies at least 1/(2d) from an integer, while the
// float product (r + 1/2) * fl(1/d) is off by under (r + 1/2) / d * 2^-23 <
// 1/(2d); truncation therefore gives q exactly.
__device__ __forceinline__ int fdivmod(int r, int d, float inv_d, int &m)
{
    const int q = __float2int_rz(__fmul_rn(__int2float_rn(r) + 0.5f, inv_d));
    m = r - q * d;
    return q;
}

// ------------------------------------------------------------------ errors
struct Error {
    pne_status st;
    std::string msg;
};

void set_error(pne_ctx *ctx, pne_status st, const std::string &msg);

#define PNE_CUDA_TRY(ctx, expr)                                                   \
    do {                                                                          \
        cudaError_t e__ = (expr);                                                 \
        if (e__ != cudaSuccess) {                                                 \
            ::pne::set_error((ctx), PNE_ECUDA,                                    \
                             std::string(#expr) + ": " + cudaGetErrorString(e__)); \
            return PNE_ECUDA;                                                     \
        }                                                                         \
    } while (0)

// After a launch whose output later launches read: a launch that was refused
// (configuration, resources) queues nothing, so the launches behind it would
// read memory nobody wrote.  Checked at once, before anything depends on it.
#define PNE_LAUNCH_CHECK(ctx) PNE_CUDA_TRY(ctx, cudaGetLastError())

// Dynamic shared memory above 48 KB for a kernel.  The limit is an attribute
// of the function, shared by every context and thread of the process, so it is
// only ever raised (under one process-wide lock): a smaller request never
// lowers it under a launch of another thread that needs more.
cudaError_t grant_dynamic_smem(const void *func, size_t bytes);

// ------------------------------------------------------------------ memory
// Device buffer owned through the context's allocator.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

pne_status dev_alloc(pne_ctx *ctx, DevBuf &b, size_t bytes, cudaStream_t s);
// small pinned host buffer for device-to-host reads of counts (per thread)
int64_t *pinned_i64(pne_ctx *ctx, size_t n);
// Host->device upload through a per-thread pinned staging region: the host data
// is copied into pinned memory and the DMA is queued on `s`, so the caller may
// release its buffer at once and no stream synchronisation is implied (a
// pageable source would synchronise the stream).  The region is recycled only
// after every copy queued out of it has completed.  Not for use inside stream
// capture (a captured copy would read the region when replayed).
pne_status upload(pne_ctx *ctx, void *dst, const void *src, size_t bytes, cudaStream_t s);
struct EnumRecord;
// the record's term-sum descriptors uploaded on s (LOOP mode records)
pne_status sum_desc_prepare(pne_ctx *ctx, EnumRecord &rec, cudaStream_t s);
// Per-thread pinned readback area `slot` of at least `bytes` (nullptr if pinned
// memory is unavailable); read after synchronising the stream of the copies.
// Slots: 0 partition records, 1 sums, 2 vacuum records, 3 shape records.
constexpr int kPinnedSlots = 4;
constexpr size_t kTraceMax = 1 << 18;   // timeline records kept per trace (later ones are dropped)
void *pinned_slot(int slot, size_t bytes);
// Pinned host buffers owned by one object at a time (batch results), from a
// per-context pool: *got receives the buffer's size; nullptr if none can be had.
void *take_pinned(pne_ctx *ctx, size_t bytes, size_t *got);
void give_pinned(pne_ctx *ctx, void *p, size_t bytes);
void dev_free(pne_ctx *ctx, DevBuf &b, cudaStream_t s);

// ------------------------------------------------------------------ shared objects
// The streams on which a device object shared by several handles (a geometry,
// an enumeration record) was used: each user, when it is destroyed, records an
// event on the stream it last used.  The object's memory is released on the
// context's release stream after it has waited for every such event, so it is
// never handed to a new allocation while a kernel queued by any user can still
// read it, whichever thread or stream drops the last reference.
// Events come from (and return to) the owning context's pool.
struct UseFence {
    std::mutex mu;
    std::vector<std::pair<cudaStream_t, cudaEvent_t>> uses;
    void note(pne_ctx *ctx, cudaStream_t s);
    // makes `target` wait for every noted use; false when a CUDA call failed
    bool join(cudaStream_t target);
    // returns the events to the context's pool (the object's destructor)
    void release(pne_ctx *ctx);
};
cudaEvent_t take_event(pne_ctx *ctx);
void give_event(pne_ctx *ctx, cudaEvent_t ev);

// ------------------------------------------------------------------ geometry
// Host + device copy of one network geometry (closed or with open bonds).
struct Geometry {
    int n_sites = 0, n_bonds = 0, n_legs = 0;
    std::vector<int32_t> bond_site, bond_dim, site_ptr, site_bonds;
    std::vector<int32_t> bond_leg;      // [n_bonds][2] leg index at each end (-1 open)
    std::vector<int32_t> inc_slot;      // [n_legs] slot whose message arrives here
    std::vector<int64_t> tens_off;      // [n_sites+1] row-major tensor offsets
    std::vector<int32_t> blk_off;       // [n_sites][64] excitation-block offsets
    std::vector<int32_t> color_ptr;     // [n_colors+1] proper colouring of the sites (closed bonds)
    std::vector<int32_t> color_sites;   // [n_sites] sites grouped by colour; within a colour by leg count, then id
    std::vector<int32_t> site_nbr;      // [n_legs][2] per leg of site_bonds: (bond, site at its other end; -1 open)
    int n_colors = 0;
    int max_deg = 0, max_dim = 0;
    uint64_t hash = 0;
    // device mirrors
    int32_t *d_bond_site = nullptr, *d_bond_dim = nullptr, *d_site_ptr = nullptr,
            *d_site_bonds = nullptr, *d_bond_leg = nullptr, *d_inc_slot = nullptr,
            *d_blk_off = nullptr, *d_color_ptr = nullptr, *d_color_sites = nullptr;
    int64_t *d_tens_off = nullptr;
    int2 *d_site_nbr = nullptr;
    DevBuf storage;
};

// ------------------------------------------------------------------ dense grid contraction
// Row-by-row contraction of a closed lx x ly grid network (dense.cu): one GEMM
// per site on a ring-ordered running tensor, on the tensor cores (TF32, BF16)
// or in FP64 on the CUDA cores.
struct SiteMap {
    int64_t t_off;          // tensor start in a set
    int64_t b_off;          // site matrix start in a set
    int stride[4];          // strides of l, u, r, d in T_v (0 for a boundary leg)
    int dim[4];             // dims of l, u, r, d (1 at a boundary)
};
struct GridStep {
    int Ku, Kh, Nd, Nh;     // up, left, down, right dims of the site
    int64_t R;              // rows of the running tensor's matrix
};
struct GridPlan {
    int n = 0;
    std::vector<SiteMap> maps;
    std::vector<GridStep> steps;
    std::vector<int64_t> ldb;   // site-matrix row stride (padded to the 16-byte unit)
    int64_t b_total = 0, max_state = 0;
};
// checks the grid (site id = y * lx + x, each neighbour pair joined by one bond)
pne_status grid_plan(pne_ctx *ctx, int lx, int ly, int n_bonds, const int32_t *bond_site, const int32_t *bond_dim,
                     const int32_t *site_ptr, const int32_t *site_bonds, const int64_t *data_off, pne_dtype dtype,
                     int nb, GridPlan &plan);
// h[2b] = mantissa, h[2b+1] = log2 scale of set b; bound = first-order relative
// rounding bound (to the absolute contraction); synchronises s
pne_status grid_run(pne_ctx *ctx, const GridPlan &plan, const double *data_dev, int64_t set_stride, int nb,
                    pne_dtype dtype, cudaStream_t s, std::vector<double> &h, double &bound);

// ------------------------------------------------------------------ handles
struct EnumRecord;  // cluster and term lists of one closed geometry
struct GeomPair;    // full + closed geometry of one network (shared, cached)

}  // namespace pne

namespace pne {
struct ProfRec {
    const char *name;
    cudaEvent_t a, b;
    cudaStream_t s;
};
struct HostRec {
    const char *name;
    double t0, t1;        // ms since the trace base
};
struct Profiler {
    std::mutex mu;
    std::atomic<bool> on{false};    // read without the lock by every launch site
    bool trace = false;             // keep every record in order (a timeline), not only the sums
    cudaEvent_t base = nullptr;     // GPU time origin of the timeline
    double host_base = 0.0;         // steady-clock ms at the origin
    std::vector<ProfRec> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<int64_t, double>> acc;
    std::vector<HostRec> host_trace;
    struct GpuRec { const char *name; cudaStream_t s; double t0, t1; };
    std::vector<GpuRec> gpu_trace;
};
}  // namespace pne

struct pne_ctx {
    pne::Profiler prof;
    int device = 0;
    int n_sm = 0;
    int64_t arena_max = 0;        // node-arena limit of the cluster search (0: the built-in limit)
    std::atomic<int> occ_expand{-1};   // resident blocks per SM of the search kernel (-1: not queried)
    pne_alloc_fn alloc = nullptr;
    pne_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
    std::map<std::string, std::shared_ptr<pne::EnumRecord>> enum_cache;
    std::map<std::string, int64_t> arena_hint;   // search-arena size that fitted, per (geometry, K, mode)
    std::map<uint64_t, std::vector<std::shared_ptr<pne::GeomPair>>> geom_cache;   // by input-array hash
    // BP launch decisions per dynamic shared-memory size: the cluster size the
    // device schedules (0: none) and the blocks per SM of the grid form
    std::map<std::pair<size_t, int>, int> bp_cluster;
    std::map<size_t, int> bp_grid_occ;
    std::mutex launch_mu;
    std::mutex cache_mu;
    // stream on which shared objects (geometries, enumeration records, batch
    // plans) are released, after waiting for every stream that used them
    cudaStream_t release_stream = nullptr;
    std::vector<cudaEvent_t> event_pool;          // timing-free events for use fences
    std::mutex event_mu;
    std::vector<std::pair<void *, size_t>> pinned_pool;   // free pinned host buffers (take_pinned)
    std::mutex pinned_mu;
    // side streams for independent launches of one call (fork/join through
    // events, serialised per context by side_mu)
    static constexpr int kSideStreams = 6;
    cudaStream_t side[kSideStreams] = {};
    cudaEvent_t side_ev[kSideStreams + 1] = {};
    bool side_ready = false;
    std::mutex side_mu;
    // streams lent to one call at a time (the shape stage of an enumeration),
    // each with a fork and a join event
    struct Lent { cudaStream_t s = nullptr; cudaEvent_t fork = nullptr, join = nullptr; };
    std::vector<Lent> stream_pool;
    std::mutex pool_mu;
};

namespace pne {
// The geometry of one network as given (full) and with its open bonds removed
// (closed), host tables plus device copies; shared by every partition of the
// same geometry through the context's cache.
struct GeomPair {
    pne_ctx *ctx = nullptr;
    Geometry full;                       // as given (may have open bonds)
    Geometry closed;                     // open bonds removed, bonds renumbered
    std::vector<int32_t> closed_of_full; // full bond id -> closed id (-1 open)
    std::vector<int32_t> open_bonds;     // full ids of open bonds, ascending
    std::vector<int32_t> open_dims;
    uint64_t key = 0;                    // hash of the input arrays
    UseFence uses;                       // streams of the partitions that used it
    cudaEvent_t ready = nullptr;         // recorded after the device copies were queued
    // gauge-transform table (open position per full bond, then the open dims)
    // and the largest site tensor, fixed by the geometry
    DevBuf gauge_tab;
    int gauge_nmax = 1;
    ~GeomPair();
};
}  // namespace pne

struct pne_partition {
    pne_ctx *ctx = nullptr;
    std::shared_ptr<pne::GeomPair> geo;
    int n_sets = 1;                  // tensor sets (n_batch)
    int n_slices = 1;                // prod of open dims
    int n_members = 1;               // n_sets * n_slices
    pne::DevBuf storage;             // one allocation holding the buffers below (views, not owners)
    pne::DevBuf T;                   // [n_sets][full.tens_off[N]] raw FP64
    pne::DevBuf msg;                 // [2][n_sets][full.n_legs][8]
    pne::DevBuf gauge;               // [n_sets][full.n_bonds][2][64] leg matrices
    pne::DevBuf Mb;                  // [n_members][closed.tens_off[N]] blocked, FP64
    pne::DevBuf site_info;           // [n_members][N] double: z_v (raw)
    pne::DevBuf site_scale;          // [n_members][N] double: 1 or 2^e for zero sites
    pne::DevBuf site_zero;           // [n_members][N] int8
    pne::DevBuf vac;                 // [n_members] {log|Zref|, sign, n_zero} as 3 doubles
    pne::DevBuf Mb32;                // FP32/TF32 copy (lazy)
    pne::DevBuf Mb16;                // BF16 copy (lazy)
    int mb32_dtype = -1;
    int arithmetic = 0;              // BP sweeps: 0 FP64, 1 float-float
    bool user_proj = false;          // projectors given by the caller (no sweeps, no convergence test)
    std::vector<int32_t> bp_iters;   // per set
    std::vector<double> bp_residual; // per set
    cudaStream_t last_stream = nullptr;
    // deferred convergence record (async_status): [res B doubles][flags 4][iters B]
    pne::DevBuf rec_dev;             // deferred convergence record (a view of storage or of rec_own)
    pne::DevBuf rec_own;             // its own buffer when an update defers a record the build did not
    bool rec_pending = false;
    pne::UseFence uses;              // streams of the terms handles that read it
};

namespace pne {

// Cluster/term lists of one closed geometry at one (K, mode).
struct EnumRecord {
    pne_ctx *ctx = nullptr;
    int K = 0, mode = 0, width = 0, vwidth = 0;
    int n_closed = 0;
    uint64_t n_clusters = 0;
    std::vector<int64_t> size_start;            // [K+2] clusters sorted by size
    DevBuf cl_edges;                            // [n][width] int32 (closed ids)
    DevBuf cl_verts;                            // [n][vwidth] int32 sorted, -1 pad
    DevBuf cl_size;                             // [n] int32
    // tuples of >= 2 clusters, one list per tuple length, sorted by order
    struct Level {
        int m = 0;
        uint64_t n = 0;
        DevBuf idx;                             // [n][m] int32
        std::vector<int64_t> order_start;       // [K+2]
    };
    std::vector<Level> levels;
    uint64_t n_terms = 0;                       // including the empty term
    std::vector<uint64_t> terms_by_order;       // [K+1]
    // per-shape contraction plans (bond dimension > 2 somewhere)
    bool shaped = false;
    int n_shapes = 0, max_out = 0;
    DevBuf shape_of;                            // [n] int32 shape id per cluster
    DevBuf perm;                                // [n] int32 clusters ordered by shape
    DevBuf plans;                               // [n_shapes][plan ints]
    DevBuf plan_steps;                          // [n_shapes] int32
    DevBuf ops;                                 // per shape: its plan's multiply-adds in order, (xi << 16) | mi
    DevBuf op_off;                              // [n_shapes + 1] int64 offsets into ops
    DevBuf step_off, step_site;                 // [n][step_stride] int32: block offset within a tensor
    int step_stride = 0;                        //   set and the site of every plan step of every cluster
    std::vector<uint64_t> shape_fma;            // [n_shapes] multiply-adds of the plan
    std::vector<int64_t> shape_count;           // [n_shapes] clusters per shape
    // perm lists the clusters by running-tensor class (largest intermediate
    // tensor of the plan, rounded up to a power of two), then by shape:
    // class q holds perm[class_start[q], class_start[q+1]) and needs class_xmax[q]
    std::vector<int64_t> class_start;
    std::vector<int> class_xmax;
    UseFence uses;                              // streams of the terms handles that used it
    // combinatorial form (COMB mode): the clusters are the distinct connected
    // components of the kept bonds of the sub-networks; each term is one
    // sub-network (order = number of active partitions).  Contractions run on
    // a virtual copy of the closed geometry whose bond dimensions are d + 1, so
    // that the excited range 1..d of the blocked layout is the full range of a
    // kept bond (blocks gathered from the gauged tensors).
    bool comb = false;
    Geometry vgeo;
    std::vector<uint64_t> empty_by_order;       // [K+1] sub-networks with no kept bond
    // the term-sum descriptors (per order, chunks of clusters and of each tuple
    // level), built on the device with the record; -1: not built
    DevBuf sum_desc;
    int n_sum_desc = -1;
    ~EnumRecord();
};

}  // namespace pne

struct pne_terms {
    pne_ctx *ctx = nullptr;
    const pne_partition *part = nullptr;
    std::shared_ptr<pne::EnumRecord> rec;
    int K = 0, mode = 0;
    int dtype = -1;                      // dtype of the last contraction
    pne::DevBuf w;                       // [n_members][n_clusters] double
    pne::DevBuf nzc;                     // [n_members][n_clusters] int32
    pne::DevBuf sums;                    // ALL mode / reduction partials
    pne::DevBuf status;                  // int32 error flags
    bool contracted = false;
    cudaStream_t last_stream = nullptr;  // stream of the last call that used the handle
    pne::DevBuf Mf, Mf32, Mf16;          // COMB: full-range blocks of the virtual geometry
    pne::DevBuf sum_done;                // [n_members] uint32 blocks finished in the term sums (zero between calls)
};

namespace pne {

// ------------------------------------------------------------------ profiling
// Records CUDA events around one launch when the context's profiler is on.
struct ProfScope {
    pne_ctx *ctx;
    cudaStream_t s;
    const char *name;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(pne_ctx *c, cudaStream_t st, const char *n);
    ~ProfScope();
};

// Host wall time of a stretch of library code, accumulated under "host:<name>"
// while profiling is on (the host side of a call: launches, allocations,
// synchronisations and host loops).
struct HostScope {
    pne_ctx *ctx;
    const char *name;
    double t0 = -1.0;
    HostScope(pne_ctx *c, const char *n);
    ~HostScope();
    void stop();          // end the stretch early (the destructor then records nothing)
};

// ------------------------------------------------------------------ kernels
// BP, gauge, blocked layout (bp.cu)
// `rec` receives the convergence record, [n_sets] residuals (f64), 4 flags
// (i32: grid-barrier timeout, zero message or overlap, 0, 0), [n_sets] sweeps
// (i32); host memory (read after the stream synchronises) or, with
// cudaMemcpyDeviceToDevice, device memory.
pne_status launch_bp(pne_ctx *ctx, pne_partition *p, double tol, int max_iter, double damping,
                     cudaStream_t s, void *rec, int arithmetic = 0,
                     cudaMemcpyKind rec_kind = cudaMemcpyDeviceToHost);
// read a deferred convergence record (synchronises the partition's stream)
pne_status partition_settle(pne_ctx *ctx, pne_partition *p);
// parse a convergence record [res B doubles][flags 4][iters B] into the partition;
// returns the BP status (ETIMEOUT, EDEGENERATE, ENOCONV or OK)
pne_status partition_record(pne_ctx *ctx, pne_partition *p, const char *rec);
pne_status launch_gauge(pne_ctx *ctx, pne_partition *p, cudaStream_t s, int32_t *h_flag);
// user projectors: the caller's rank-1 projector vectors placed as the final
// messages (no sweeps), then the gauge pairs; the convergence record (zeros,
// the gauge's degenerate flag) copied to rec like launch_bp's
pne_status launch_user_projectors(pne_ctx *ctx, pne_partition *p, const double *user_u, const double *user_v,
                                  cudaStream_t s, void *rec, cudaMemcpyKind rec_kind);
pne_status launch_convert(pne_ctx *ctx, pne_partition *p, int dtype, cudaStream_t s);
// FP64 -> FP32 (TF32 rounding for PNE_TF32) or BF16 copy of n entries
pne_status convert_buffer(pne_ctx *ctx, const double *src, int64_t n, int dtype, void *dst, cudaStream_t s);

// enumeration (enumerate.cu)
pne_status enumerate_clusters(pne_ctx *ctx, const Geometry &g, int K, int mode,
                              EnumRecord &rec, cudaStream_t s);
pne_status enumerate_tuples(pne_ctx *ctx, EnumRecord &rec, cudaStream_t s);
// The same in two halves: the first round's counting with its readback queued
// (begin), then the wait, its writing pass and any further rounds (finish).
struct TuplePrep {
    bool active = false;          // a round's counting is queued
    int m = 1, s_min = 0;         // length of the round's input tuples; smallest cluster size
    int64_t n_in = 0, n_units = 0;
    std::vector<int64_t> size_end;
    DevBuf d_size_end, in_idx, in_ord, uoff, counts, base;
    bool in_owned = true;
    int64_t *h = nullptr;         // pinned readback of the (order, unit) row starts
    size_t tsmem = 0;
};
pne_status tuples_begin(pne_ctx *ctx, EnumRecord &rec, TuplePrep &tp, cudaStream_t s);
pne_status tuples_finish(pne_ctx *ctx, EnumRecord &rec, TuplePrep &tp, cudaStream_t s);
// Releases the buffers of an unfinished TuplePrep (stream-ordered on `s`).
void tuples_abort(pne_ctx *ctx, TuplePrep &tp, cudaStream_t s);

// contraction and sums (contract.cu)
pne_status launch_contract(pne_ctx *ctx, pne_terms *t, int dtype, cudaStream_t s);
// a device-to-host copy queued with the sums' read-back (after their kernels,
// so that it does not sit between the contraction and the sums on the stream)
struct D2HCopy {
    void *dst;
    const void *src;
    size_t bytes;
};
pne_status launch_sums(pne_ctx *ctx, const pne_terms *t, cudaStream_t s,
                       std::vector<double> &c, std::vector<double> &abs_c, int32_t *h_status,
                       const std::vector<D2HCopy> &extra = {});
pne_status launch_all_mode(pne_ctx *ctx, pne_terms *t, int dtype, cudaStream_t s);
pne_status launch_plan_work(pne_ctx *ctx, const pne_terms *t, cudaStream_t s, uint64_t *fma);
// device tables of a geometry built from its bond_site/bond_dim/site_ptr/site_bonds (pne_api.cu)
pne_status finish_geometry(pne_ctx *ctx, Geometry &g, cudaStream_t s);
// contraction plans per cluster shape, in two halves around a synchronisation
struct ShapePrep {
    DevBuf dh;                    // per-cluster hashes on the device
    void *h_pinned = nullptr;     // their readback
    bool active = false;
    // after shapes_plan: shape ids and representatives, the verification and
    // plan launches, and their queued readback
    bool planned = false;
    std::vector<int32_t> shape, rep, bad, stats;
    DevBuf dshape, drep, dbad, dstats;
    char *hp = nullptr;
    size_t nb = 0;
    int ns = 0;
};
void shapes_release(pne_ctx *ctx, ShapePrep &sp, cudaStream_t s);
bool shapes_needed(const Geometry &g, const EnumRecord &rec);
// Shape preparation in three stages on one stream, each queueing work and
// readbacks without waiting except for the readback of the stage before:
// hashes (begin), shape ids + plans (plan), multiply-add lists and cluster
// order (complete).  shapes_finish = plan + complete.
pne_status shapes_begin(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s);
pne_status shapes_plan(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s);
pne_status shapes_complete(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s);
pne_status shapes_finish(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s);
pne_status launch_convert_only(pne_ctx *ctx, const pne_partition *p, int dtype, cudaStream_t s);

// batched form (contract.cu)
struct BatchPlan;
pne_status batch_plan_create(pne_ctx *ctx, const std::vector<pne_terms *> &terms, int dtype, cudaStream_t s,
                             BatchPlan **out);
pne_status batch_prepare(pne_ctx *ctx, BatchPlan *bp, int wpb, int bps, cudaStream_t s);
pne_status batch_enqueue(pne_ctx *ctx, BatchPlan *bp, int wpb, int bps, int sched, cudaStream_t s);
int batch_max_blocks_per_sm(BatchPlan *bp, int wpb);
// releases the plan's buffers behind the work queued on `s` (its last stream)
void batch_plan_destroy(pne_ctx *ctx, BatchPlan *bp, cudaStream_t s);
double *batch_host_out(BatchPlan *bp);
const std::vector<int64_t> &batch_out_offsets(BatchPlan *bp);
int32_t batch_status_host(BatchPlan *bp);

// result assembly shared by pne_sum and pne_batch_run
void finalize_result(pne_result &r, int K, int mode, int dtype, const double *c, const double *abs_c,
                     const double *vac, uint64_t n_terms, uint64_t n_clusters, int bp_iters, double bp_residual);
pne_status launch_fma_peak(pne_ctx *ctx, int dtype, cudaStream_t s, double *flops);

// exclusive scan of int64 counts on the device; total returned on the host
pne_status device_exclusive_scan(pne_ctx *ctx, int64_t *d_counts, int64_t n, int64_t *h_total,
                                 cudaStream_t s);
pne_status device_exclusive_scan_to(pne_ctx *ctx, int64_t *d, int64_t n, int64_t *d_total, cudaStream_t s);

}  // namespace pne
