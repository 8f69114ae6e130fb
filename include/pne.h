/*
 * pne.h -- C ABI of the GB300 partitioned-network-expansion (PNE) library.
 *
 * The library evaluates the truncated linear form of the partitioned network
 * expansion (Evenbly, Gray & Chan, "Partitioned Expansions for Approximate
 * Tensor Network Contractions", Sec. II.A, Eq. A2-A4) with every bond
 * partitioned by a rank-1 projector built from belief-propagation messages
 * (Sec. II.B, Eq. A7, symmetrised as in App. B).  A term is the network with
 * Q = I - P on a set E of bonds and P on the rest; it factorises into the
 * capped sites and one local contraction per connected cluster of E.  Terms
 * of order |E| <= K are summed with unit weights; higher orders and the
 * residue (Eq. res) are neglected.
 *
 * Conventions shared by every call
 *   - Every call returns a pne_status; none aborts the process.  After an
 *     error, pne_last_error(ctx) holds a one-line message (per thread).
 *   - Inputs are borrowed for the duration of the call and copied.
 *   - Handles (pne_ctx, pne_partition, pne_terms) are owned by the caller once
 *     returned and released with the matching *_destroy call; device memory
 *     they hold is released there, stream-ordered behind the work already
 *     queued for the handle (on every stream that used it), so a handle may be
 *     destroyed while that work is still running.  Destroy batches before the
 *     terms handles they hold, and terms handles before the partition they
 *     were enumerated from.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it unless stated otherwise.
 *   - One context serves one device.  It may be used by several host threads
 *     at once, provided each handle (partition, terms, batch) is used by one
 *     thread at a time: the context's shared state -- the geometry and
 *     enumeration caches, launch decisions, stream and event pools, the
 *     profiler -- is guarded, and objects shared between handles (a cached
 *     geometry or enumeration) are released only after every stream that used
 *     them.  pne_ctx_set_allocator and pne_ctx_destroy must not overlap any
 *     other call on the context.
 *   - Floating point: partitions (messages, gauge, site values) are FP64;
 *     cluster contractions run in the pne_dtype given; term products and the
 *     per-order sums are FP64.
 */
#ifndef PNE_H
#define PNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pne_ctx pne_ctx;             /* device, allocator, enumeration cache */
typedef struct pne_partition pne_partition; /* messages, gauged site tensors, z_v  */
typedef struct pne_terms pne_terms;         /* clusters, terms, cluster values     */

typedef enum {
    PNE_OK = 0,
    PNE_EINVAL = 1,       /* malformed input or unsupported size              */
    PNE_ENOMEM = 2,       /* device or host allocation failed                 */
    PNE_ECUDA = 3,        /* a CUDA runtime call failed                       */
    PNE_ENOCONV = 4,      /* BP did not reach tol within max_iter sweeps      */
    PNE_EDEGENERATE = 5,  /* |<m_s0|m_s1>| below 1e-300 on some bond, or a
                             message of zero norm                             */
    PNE_ETIMEOUT = 6,     /* a bounded device-side wait gave up               */
    PNE_EOVERFLOW = 7,    /* a per-cluster or per-term buffer limit exceeded  */
    PNE_EBUSY = 8         /* resource in use (e.g. scratch of another call)   */
} pne_status;

typedef enum { PNE_F64 = 0, PNE_F32 = 1, PNE_TF32 = 2, PNE_BF16 = 3 } pne_dtype;
/* LOOP: clusters with a site of cluster-degree one ("dangling excitation",
 *       Sec. III.A) are dropped -- they vanish at a BP fixed point.
 * ALL:  every bond subset is a term (networks with <= 30 closed bonds).
 * COMB: the combinatorial form over multi-index partitions (handles made by
 *       pne_enumerate_combinatorial only). */
typedef enum { PNE_MODE_LOOP = 0, PNE_MODE_ALL = 1, PNE_MODE_COMB = 2 } pne_mode;

/* Library limits (checked; violations return PNE_EINVAL). */
#define PNE_MAX_DEG 6        /* legs per site                                */
#define PNE_MAX_DIM 8        /* bond dimension                               */
#define PNE_MAX_ORDER 32     /* expansion order K                            */

/*
 * A network of tensors (Eq. A1).  Sites 0..n_sites-1, bonds 0..n_bonds-1.
 *   bond_site  [n_bonds][2] host: the two sites of each bond; the second is -1
 *              for an open index (Sec. III.D).  No bond joins a site to itself.
 *   bond_dim   [n_bonds] host: index dimension, 2..PNE_MAX_DIM.
 *   site_ptr   [n_sites+1], site_bonds [site_ptr[n_sites]] host: each site's
 *              legs = its bonds in ascending bond id (CSR).
 *   data       site tensors, FP64, row-major over the site's legs in the order
 *              above; n_batch consecutive tensor sets of identical geometry,
 *              set b at data + b * data_off[n_sites].  Host pointer, or device
 *              pointer when data_on_device != 0.
 *   data_off   [n_sites+1] host: start of each site's tensor within a set.
 */
typedef struct {
    int32_t n_sites, n_bonds;
    const int32_t *bond_site;
    const int32_t *bond_dim;
    const int32_t *site_ptr, *site_bonds;
    const double *data;
    const int64_t *data_off;
    int32_t data_on_device;
    int32_t n_batch;
} pne_network;

/* BP options (the paper leaves the schedule open): sweeps from the uniform
 * message 1/sqrt(d) in colour order (the sites of one colour of a greedy
 * proper colouring update together from the latest messages: red-black on
 * bipartite lattices); each message normalised to unit 2-norm with its
 * largest-magnitude entry positive; stop when the largest entry change in a
 * sweep is below tol.  The fixed point is the one Jacobi sweeps reach.
 * damping in [0,1) mixes the previous message in. */
typedef struct {
    double tol;          /* default 1e-13 when <= 0 */
    int32_t max_iter;    /* default 10000 when <= 0 */
    double damping;      /* default 0 */
    int32_t arithmetic;  /* the BP sweeps and the gauge transform of the site
                            tensors in 0: FP64, 1: float-float (pairs of FP32
                            with error-free sums and products, ~2^-48 relative
                            precision per operation, on the FP32 pipes); the
                            messages, projectors and blocked tensors handed on
                            are FP64 either way */
    int32_t async_status; /* 0: pne_build_partition synchronises its stream and
                            returns the convergence status; 1: it returns once
                            the work is queued (no synchronisation), and the
                            convergence record is read by the next call that
                            synchronises for this partition (pne_sum returns
                            PNE_ENOCONV / PNE_EDEGENERATE / PNE_ETIMEOUT then,
                            after writing every result; non-converged sets show
                            bp_iters == 0) */
    /* User projectors instead of BP (Eq. A2: P_b may be any projector; the
     * identities of Eq. A3-A4 hold for every choice).  With
     * use_user_projectors = 1, closed bond b = (s0, s1) (s0 = bond_site[b][0])
     * takes the rank-1 projector
     *     P_b[a0][a1] = u_b[a0] v_b[a1] / (u_b . v_b),
     * a0 the index on s0's side, a1 on s1's, and Q_b = I - P_b.  user_u and
     * user_v hold, for every tensor set and then every closed bond in id order,
     * bond_dim[b] FP64 entries each ([n_batch][sum of closed bond dimensions],
     * host memory, read during the call; open bonds take none).  No sweeps run
     * (bp_iters = 0, residual 0, never PNE_ENOCONV); tol, max_iter and damping
     * are ignored; |u_b . v_b| < 1e-300 or u_b = 0 gives PNE_EDEGENERATE. */
    int32_t use_user_projectors;
    const double *user_u;
    const double *user_v;
} pne_partition_opts;

typedef struct {
    int32_t max_order;   /* K: keep terms with |E| <= K                      */
    int32_t mode;        /* pne_mode                                          */
    int32_t use_cache;   /* reuse a cached enumeration of the same geometry  */
    int32_t max_cluster; /* keep only clusters of at most this many bonds
                            (terms still up to order max_order, built from
                            those clusters); 0 or >= max_order: no cap       */
} pne_enum_opts;

/* Result for one network (one tensor set, one open-index assignment). */
typedef struct {
    int32_t sign;            /* sign of Z_K                                   */
    double log_abs;          /* ln|Z_K|                                       */
    double value;            /* Z_K as a double (+-inf when out of range)     */
    double c[PNE_MAX_ORDER + 1];     /* c_k = (sum of order-k terms) / Z_ref  */
    double abs_c[PNE_MAX_ORDER + 1]; /* same with |term|                      */
    int32_t n_orders;        /* K + 1                                         */
    double log_abs_zref;     /* ln|Z_ref|, Z_ref = prod of nonzero z_v        */
    int32_t sign_zref;
    int32_t n_zero_sites;    /* sites with z_v == 0                            */
    double log_series;       /* ln|Z_ref| + sum_{k=1..K} [x^k] ln(sum_j c_j x^j);
                                NaN when undefined (not part of the paper)    */
    double err_bound;        /* a-priori rounding bound on Z_K, relative:
                                (gamma(2(K+1)) u_dtype sum_{k}|c_k|' +
                                gamma(K + 2 + log2 n_terms) 2^-53 sum_k|c_k|)
                                / |sum_k c_k|, where ' leaves out the exact
                                empty term, gamma(n) = n u / (1 - n u) and
                                u_dtype = 2^-53, 2^-24, 2^-11, 2^-8 for F64,
                                F32, TF32, BF16                               */
    uint64_t n_terms, n_clusters;
    int32_t bp_iters;        /* sweeps BP took for this tensor set            */
    double bp_residual;      /* last sweep's largest message change           */
} pne_result;

/* ---- context ------------------------------------------------------------ */
pne_status pne_ctx_create(int device, pne_ctx **out);
void pne_ctx_destroy(pne_ctx *ctx);
const char *pne_last_error(pne_ctx *ctx);

/* Optional device allocator (e.g. a framework's caching allocator).  Without
 * one the library uses cudaMallocAsync / cudaFreeAsync on the call's stream. */
typedef void *(*pne_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*pne_free_fn)(void *ptr, size_t bytes, void *stream, void *user);
pne_status pne_ctx_set_allocator(pne_ctx *ctx, pne_alloc_fn alloc, pne_free_fn free_fn, void *user);

/* ---- the four calls of the hot path ------------------------------------- */

/* Build the bond partitions (Sec. II.B, Eq. A7, App. B): BP to a fixed point
 * (boundary reflection on open indices, Sec. III.D), normalise each bond's
 * messages to unit overlap, gauge every closed bond so that P = e0 e0^T and
 * Q = diag(0,1,..,1), and keep the gauged site tensors, z_v and the vacuum
 * value on the device.  Synchronises `stream` once at the end to read the
 * convergence record (unless opts->async_status: see pne_partition_opts).
 * Returns PNE_ENOCONV (handle still returned, usable) when some tensor set
 * did not converge, PNE_EDEGENERATE on a zero overlap. */
pne_status pne_build_partition(pne_ctx *ctx, const pne_network *net,
                               const pne_partition_opts *opts, void *stream,
                               pne_partition **out);
void pne_partition_destroy(pne_partition *p);

/* Enumerate the clusters (connected bond sets with |C| <= K, LOOP or ALL
 * mode) and the terms (vertex-disjoint cluster tuples with total size <= K,
 * Eq. A4).  Geometry only: the lists are shared by every tensor set and
 * cached in the context when use_cache != 0.  Synchronises `stream` while it
 * searches (the counts size the buffers).  The contraction plans of the
 * clusters are prepared on a second stream lent from the context (created at
 * the device's highest stream priority) and joined back into `stream` before
 * the call returns.  With use_cache != 0 the returned lists and buffers are
 * complete on return and may be used from any stream; with use_cache == 0
 * their last writes are still queued on `stream`, so use them on `stream` or
 * after it (an event or a synchronisation).  n_clusters / n_terms may be
 * NULL. */
pne_status pne_enumerate_terms(pne_ctx *ctx, const pne_partition *part,
                               const pne_enum_opts *opts, void *stream,
                               pne_terms **out, uint64_t *n_clusters, uint64_t *n_terms);
void pne_terms_destroy(pne_terms *t);

/* The combinatorial form of the expansion over multi-index partitions
 * (Sec. II.A Eq. A6; Sec. II.C Eq. A8-A10).  Partition p transects the bonds
 * partition_bonds[partition_ptr[p] .. partition_ptr[p+1]) (ids of the network
 * as given; closed bonds only; two partitions may share a bond), and its
 * projector is the product of the rank-1 BP projectors of those bonds (Eq.
 * A10, from `part`).  The terms are the 2^M - 1 sub-networks Z(P^x), x a
 * non-empty set of partitions: every bond of an active partition cut and
 * capped by the messages, every other bond kept at its full dimension.  A
 * sub-network factorises into the connected components of its kept bonds
 * (sites with no kept bond contribute their capped value z_v); the handle
 * lists the distinct components as its clusters, pne_contract_terms contracts
 * each exactly, and pne_sum forms every sub-network as the product of its
 * components and sums them by |x|:
 *   c_k = sum_{|x| = k} Z(P^x) / Z_ref  (k = 1..M, c_0 = 0),
 *   Z   = Z_ref sum_{k=1..M} (-1)^{k+1} c_k,
 * the residue Z(Q_1, ..., Q_M) neglected (log_series is NaN).  Limits: M <=
 * 20; every component of at most 32 bonds and 32 sites; bond dimensions <= 7
 * (PNE_EINVAL otherwise).  A component whose contraction needs a running
 * tensor above the kernels' limit makes pne_sum return PNE_EOVERFLOW.
 * Synchronises `stream`.  n_components / n_terms may be NULL. */
pne_status pne_enumerate_combinatorial(pne_ctx *ctx, const pne_partition *part, int32_t n_partitions,
                                       const int32_t *partition_ptr, const int32_t *partition_bonds, void *stream,
                                       pne_terms **out, uint64_t *n_components, uint64_t *n_terms);

/* Contract every cluster of every tensor set in `dtype` (Sec. II.C: with P
 * bonds cut and capped, a term factorises into the capped sites and one
 * local contraction per connected excited cluster; Sec. III.A: that
 * contraction is the cluster's only cost): w(C) = Z'_C /
 * prod_{v in C, z_v != 0} z_v with a per-cluster power-of-two exponent carried
 * through the contraction.  Asynchronous. */
pne_status pne_contract_terms(pne_ctx *ctx, pne_terms *t, pne_dtype dtype, void *stream);

/* Form every term's value (product of its clusters' w; a term of the
 * expansion Eq. A4 is a vertex-disjoint set of clusters) and sum by order in
 * FP64 with a fixed reduction tree, keeping the orders |E| <= K (the
 * truncation of Sec. II.B); write one pne_result per tensor set and
 * open-index assignment into out[] (pne_terms_n_results entries, set-major,
 * assignments row-major over the open bonds in ascending id).  Synchronises
 * `stream`. */
pne_status pne_sum(pne_ctx *ctx, const pne_terms *t, void *stream, pne_result *out);

/* Number of pne_result entries pne_sum writes (= n_batch * prod of open dims). */
int64_t pne_terms_n_results(const pne_terms *t);

/* Open-index output (Sec. III.D: open indices are left unpartitioned, and the
 * result is the network's tensor over them; Eq. B2 measures its error).  The
 * entry at one assignment o of the open indices is Z_K of the closed slice
 * with the open indices fixed to o (the slices share the partition's
 * projectors and the enumeration).  Runs pne_sum's work on `stream`
 * (synchronises it) and writes, for every tensor set b,
 *   tensor[b][o] = out[b * n_open + o] * exp(log_scale[b]),
 * o row-major over the open bonds in ascending bond id, n_open = the product
 * of their dimensions (pne_terms_n_results(t) / n_batch), and log_scale[b] =
 * max_o ln|Z_K(b, o)| so that |out| <= 1 and no entry overflows (log_scale is
 * -inf and out zero when every slice of the set is zero).
 *   out        host [n_batch * n_open] doubles, caller-owned
 *   log_scale  host [n_batch] doubles, caller-owned
 * A network without open indices gives one entry per set (its Z_K). */
pne_status pne_open_tensor(pne_ctx *ctx, const pne_terms *t, void *stream, double *out, double *log_scale);

/* The assembly step of pne_open_tensor alone, from results pne_sum wrote
 * (res[n_sets * n_open], set-major): host arithmetic only, no device. */
pne_status pne_open_tensor_assemble(const pne_result *res, int64_t n_sets, int64_t n_open, double *out,
                                    double *log_scale);

/* Copy the cluster list and the contracted cluster values to host memory, for
 * inspection and element-by-element checks.  LOOP and COMB modes.
 *   edges  [n_clusters][max_order] int32: each cluster's bond ids (ids of the
 *          network as given), ascending, padded with -1; may be NULL.
 *   w      [pne_terms_n_results][n_clusters] double: w(C) per tensor set and
 *          open-index assignment (needs pne_contract_terms first); may be NULL.
 * Clusters are listed grouped by size.  For a combinatorial handle (COMB
 * mode) the clusters are its components and each row of `edges` holds
 * PNE_MAX_ORDER entries instead of max_order.  Synchronises `stream`. */
pne_status pne_terms_export(pne_ctx *ctx, const pne_terms *t, void *stream, int32_t *edges, double *w);

/* Re-run the partition of an existing handle on new tensors of the same
 * geometry and batch size (BP, gauge, blocked tensors), reusing its device
 * buffers, so that enumerations and batches built on the handle stay valid.
 * `data` holds n_batch tensor sets laid out as in pne_network; host pointer,
 * or device pointer when data_on_device != 0.  Synchronises `stream`. */
pne_status pne_partition_update(pne_ctx *ctx, pne_partition *p, const double *data, int32_t data_on_device,
                                const pne_partition_opts *opts, void *stream);
/* With opts->async_status != 0 the update returns without synchronising: the
 * convergence record stays on the device and is read by the next pne_sum,
 * pne_batch_run, pne_batch_create or pne_partition_update that involves the
 * partition (pne_batch_run reads the records of all its partitions together
 * and returns the first non-OK record status after writing the results).
 * Work on another stream that uses the partition must wait for `stream`
 * (an event), as with any stream-ordered call. */

/* ---- batched form: one persistent launch over many networks -------------- */

/* A batch fuses the cluster contractions (pne_contract_terms) and the term
 * sums (pne_sum) of many handles -- networks of different sizes and bond
 * dimensions, each with its own partition -- into one persistent kernel that
 * takes work from a single queue (Sec. II.D: every term can be evaluated in
 * parallel).  Contraction items of a handle come before its sum items; a sum
 * item waits (bounded) for its handle's contractions.  The launch sequence
 * (dtype conversion, fused kernel, per-order reduction, copy of the results)
 * is captured once in a CUDA graph and replayed by pne_batch_run. */
typedef struct pne_batch pne_batch;

typedef struct {
    int32_t warps_per_block;   /* 0: autotune (with blocks_per_sm)            */
    int32_t blocks_per_sm;     /* 0: autotune                                 */
    int32_t use_graph;         /* capture and replay a CUDA graph             */
    int32_t schedule;          /* order of the contraction items in the queue,
                                  with a given launch shape: PNE_SCHED_HANDLE
                                  or PNE_SCHED_LARGEST_FIRST; tuned together
                                  with the shape when autotuning              */
} pne_batch_opts;

/* Work orders of the contraction items (the sum items always follow them).
 * HANDLE: handle by handle, tensor set by tensor set, clusters in list order.
 * LARGEST_FIRST: items with the largest running tensors first (stable), so the
 * costly items do not start last and leave the tail of the launch to a few
 * warps.  Results do not depend on the order. */
#define PNE_SCHED_HANDLE 0
#define PNE_SCHED_LARGEST_FIRST 1

/* terms[i] must be LOOP-mode handles whose partitions stay alive as long as
 * the batch.  Autotuning times each candidate (launch shape, schedule) on this
 * batch and caches the winner (in memory, and in the file named by the
 * environment variable PNE_AUTOTUNE_CACHE when set).  PNE_EINVAL for a given
 * shape that does not fit or an unknown schedule.  Synchronises `stream`. */
pne_status pne_batch_create(pne_ctx *ctx, int32_t n, pne_terms *const *terms, pne_dtype dtype,
                            const pne_batch_opts *opts, void *stream, pne_batch **out);
/* Replay: writes sum_i pne_terms_n_results(terms[i]) results, handle-major.
 * Synchronises `stream`. */
pne_status pne_batch_run(pne_ctx *ctx, pne_batch *b, void *stream, pne_result *out);
int64_t pne_batch_n_results(const pne_batch *b);
/* Chosen launch shape and its timed duration (ms) from the autotuner. */
pne_status pne_batch_config(const pne_batch *b, int32_t *warps_per_block, int32_t *blocks_per_sm, double *tuned_ms);
/* Chosen work order (PNE_SCHED_*). */
pne_status pne_batch_schedule(const pne_batch *b, int32_t *schedule);
void pne_batch_destroy(pne_batch *b);

/* ---- served form: continuous batching of requests ------------------------- */

/* A server owns worker threads on the context's device.  Requests (one network,
 * any size, bond dimension and order) are admitted in arrival order while the
 * estimated device bytes of the admitted-but-unfinished requests stay within
 * device_budget_bytes and their number within max_inflight.  Admitted
 * requests are prepared concurrently (partition, enumeration -- the latter
 * from the context's geometry cache when present) on n_prep_streams streams;
 * a launcher merges every prepared request into the next fused persistent
 * launch (see pne_batch_*) while later arrivals keep being prepared, so work
 * of different requests overlaps on the device.  A request's result does not
 * depend on which other requests share its launch.  Clusters, partitions and
 * cluster values stay on the device until the request completes. */
typedef struct pne_server pne_server;

typedef struct {
    uint64_t device_budget_bytes;   /* admission limit (0: 8 GiB)              */
    int32_t max_inflight;           /* admitted, unfinished requests (0: 256)  */
    int32_t n_prep_streams;         /* preparing threads/streams (0: 4)        */
    int32_t max_batch;              /* requests per fused launch (0: 256)      */
    int32_t dtype;                  /* pne_dtype of the cluster contractions   */
    int32_t warps_per_block;        /* fused-launch shape (0: 4)               */
    int32_t blocks_per_sm;          /* (0: 2)                                  */
} pne_server_opts;

typedef struct {
    double t_arrival, t_admit, t_ready, t_done;  /* seconds since server start */
    uint64_t device_bytes;                        /* admission estimate        */
    int32_t batch_size;                           /* requests in its launch    */
} pne_request_info;

pne_status pne_server_create(pne_ctx *ctx, const pne_server_opts *opts, pne_server **out);
/* Copies the network (host tensors; n_batch must be 1, no open indices) and
 * queues it; returns at once with the request id.  A served request's
 * partition is built with float-float BP sweeps (pne_partition_opts
 * arithmetic 1, tol 1e-13). */
pne_status pne_server_submit(pne_server *s, const pne_network *net, int32_t max_order, uint64_t *id);
/* PNE_OK and the result when the request is done (its record is then
 * released), PNE_EBUSY while it is queued or running, PNE_EINVAL for an
 * unknown id; a request that failed returns its error status. */
pne_status pne_server_poll(pne_server *s, uint64_t id, pne_result *out, pne_request_info *info);
/* Blocks until every submitted request is done. */
pne_status pne_server_drain(pne_server *s);
/* Largest admitted estimate seen at once, and the server clock (seconds). */
pne_status pne_server_stats(pne_server *s, uint64_t *peak_inflight_bytes, double *now);
/* The error text of the first request that failed ("" while none has): the
 * message of the failing library call, as pne_last_error gives it in the
 * server thread that made it.  Valid until the server is destroyed. */
const char *pne_server_first_error(pne_server *s);
void pne_server_destroy(pne_server *s);

/* ---- rank-r projectors by weight passing ---------------------------------- */

/* Weight passing (App. C): a diagonal matrix of positive weights S_i on every
 * bond, found by repeated local updates that are pure changes of gauge (Eq.
 * weight1-3): for bond i between tensors A and B, the weights of all other
 * legs are absorbed into A and B, the SVDs of both (between index i and the
 * rest) and of S_A V_A^T S_i U_B S_B are taken, A and B are re-gauged and S_i
 * becomes S_C^alpha.  Sweeps visit the bonds in id order until the largest
 * weight change is below tol.  The weights are rescaled to a largest entry of
 * 1 after each update and the factor kept in a log scale.  The handle keeps,
 * on the device, the weighted network -- sqrt(S_i) absorbed into both ends of
 * every bond, so that it contracts to the input's value times exp(-log_scale)
 * -- in which the rank-r projector onto the r largest weights of a bond is the
 * restriction of its index to the first r values (the weights are sorted).
 *   net    closed network (no open indices), host or device tensors, n_batch
 *          tensor sets; every bond dimension at most 16 and at most the
 *          product of the other dimensions of either of its tensors.
 *   alpha  in (0, 1] (the paper's benchmarks use 0.8); tol > 0; max_sweeps > 0.
 * FP64 throughout.  Synchronises `stream`.  Returns PNE_ENOCONV (handle
 * still returned) when some set did not reach tol, PNE_EDEGENERATE when a
 * tensor is rank-deficient across a bond (a zero singular value). */
typedef struct pne_weights pne_weights;
pne_status pne_weight_passing(pne_ctx *ctx, const pne_network *net, double alpha, double tol, int32_t max_sweeps,
                              void *stream, pne_weights **out);
/* weights [n_batch][n_bonds][16] (zero-padded, descending per bond), sweeps
 * [n_batch], log_scale [n_batch]; host arrays, each may be NULL.  Synchronises. */
pne_status pne_weights_read(pne_ctx *ctx, const pne_weights *w, void *stream, double *weights, int32_t *sweeps,
                            double *log_scale);
void pne_weights_destroy(pne_weights *w);

/* The expansion with rank-r projectors (Sec. V.A) built on the weights: every
 * partition's projector keeps the `rank` largest weights of each of its bonds
 * (first `rank` index values of the weighted network), Q = I - P.
 *   form 0  linear form over single-index partitions (Eq. A4): terms
 *           Z(Q_1, ..., Q_k, P_{k+1}, I, ...), k = 0 .. M-1, each partition
 *           exactly one bond;
 *   form 1  combinatorial form over multi-index partitions (Eq. A6): the
 *           2^M - 1 sub-networks Z(P^x) with alternating signs.
 * Every term is the weighted network with each bond's index restricted to
 * the P range [0, rank), the Q range [rank, d) or left whole, contracted
 * exactly in FP64 (a dense contraction site by site); the residue is
 * neglected.  One pne_result per tensor set in out[n_batch]: value, sign,
 * log_abs (the scale included), c[k] = sum of the order-k terms times
 * exp(-log_scale) (k = |x| for form 1, k = position in Eq. A4 for form 0),
 * n_terms.  Partition bonds as in pne_enumerate_combinatorial.  Limits: M <=
 * 20, 1 <= rank < every partitioned bond's dimension, an intermediate tensor
 * of at most 2^20 entries (PNE_EINVAL otherwise).  Synchronises `stream`. */
pne_status pne_rank_r_expand(pne_ctx *ctx, const pne_weights *w, int32_t rank, int32_t form, int32_t n_partitions,
                             const int32_t *partition_ptr, const int32_t *partition_bonds, void *stream,
                             pne_result *out);

/* ---- infinite lattices: the strip expansion ------------------------------ */

/* Free energy density of an infinite, translation-invariant square-lattice
 * network of one tensor A (Sec. IV.C).  A partition is the set of bonds cut
 * by every L-th vertical line at one offset (L of them), or by every L-th
 * horizontal line (L more); its projector is the rank-1 BP projector on
 * every cut bond (Eq. A7, A8), which splits the lattice into strips whose
 * cut legs are capped by the BP messages (scaled to unit overlap on every
 * bond).  The expansion is the combinatorial form (Eq. A6) over the 2L
 * partitions of one L x L cell, written per cell: every non-empty subset x
 * contributes (-1)^{|x|+1} times its pieces over the cell --
 *   vertical offsets V only:   prod over the gaps w of V of lambda_w^L,
 *   horizontal offsets H only: prod over the gaps h of H of gamma_h^L,
 *   both:                      prod over w, h of Z_wh,
 * (gaps taken cyclically, summing to L) -- and f = -ln(sum) / L^2 per site
 * (two_d = 0: vertical strips only, L partitions, f = -ln(sum) / L).
 * lambda_k (gamma_k) is the leading eigenvalue of the row transfer matrix
 * of a vertical (horizontal) strip k sites wide, Z_wh the value of a capped
 * patch of w columns and h rows.  For L = 2 the sum is the paper's
 * 2 lambda_2 - lambda_1^2 (1D) and R1 - R2 + R3 - R4 (2D); the width-3 sum is
 * taken with the alternating signs of Eq. A6.
 *
 *   chi        bond dimension, 2 .. PNE_STRIP_MAX_CHI.
 *   n_tensors  1 .. 65535 tensors evaluated independently (e.g. a temperature sweep).
 *   A          [n_tensors][chi^4] doubles, each row-major over the legs
 *              [l, u, r, d] (towards x - 1, y - 1, x + 1, y + 1); host memory
 *              (A_on_device = 0) or device memory.
 *   opts       L in 1 .. PNE_STRIP_MAX_L with chi^(L+1) <= 2^28; tolerances
 *              and iteration limits (0 selects the default given beside each).
 *   out        [n_tensors] host results.
 * Method: uniform BP to bp_tol (parallel updates, FP64); each lambda_k by
 * power iteration from the product of the incoming messages, the row
 * transfer matrix applied site by site (FP64 multiply-adds) and the estimate
 * the Rayleigh quotient, until lambda changes by less than eig_tol
 * (relative) in three successive iterations (and at least L iterations, whose first L
 * iterates, closed with the outgoing messages, give Z_k1 .. Z_kL); the 2^(2L)
 * - 1 terms are summed as sign * expm1(ln term - L^2 ln z_BP) in double-double
 * arithmetic (the signs sum to one).  Needs 2 (chi^L + chi^(L+1)) doubles of
 * device memory per tensor in flight (tensors are processed in groups that fit
 * a 24 GB working set).  Returns PNE_ENOCONV (results filled with the last
 * estimates) when BP or a power iteration did not converge, PNE_EDEGENERATE
 * when a message overlap vanishes or an eigenvalue estimate or the sum is not
 * positive, PNE_EINVAL on bad arguments (nothing launched).  Synchronises
 * `stream`. */
#define PNE_STRIP_MAX_L 12
#define PNE_STRIP_MAX_CHI 8
typedef struct {
    int32_t L;               /* strip width                                   */
    int32_t two_d;           /* 1: vertical and horizontal strips; 0: vertical */
    double bp_tol;           /* largest message change (0: 1e-14)             */
    double eig_tol;          /* relative change of lambda (0: 1e-14)          */
    int32_t bp_max_iter;     /* (0: 100000)                                   */
    int32_t eig_max_iter;    /* power iterations per eigenvalue (0: 20000)    */
    int32_t arithmetic;      /* row transfer products: 0 FP64 multiply-adds,
                                1 float-float (compensated FP32 dot products,
                                ~2^-48 relative per site; FP64 storage of the
                                iterates, FP64 reductions and sums)           */
} pne_strip_opts;

typedef struct {
    double f;                /* free energy per site of A's lattice           */
    double f_bp;             /* -ln z_BP                                      */
    double log_lambda[PNE_STRIP_MAX_L + 1];  /* [k] = ln lambda_k, k = 1..L   */
    double log_gamma[PNE_STRIP_MAX_L + 1];   /* [k] = ln gamma_k (2D only)    */
    double log_z[(PNE_STRIP_MAX_L + 1) * (PNE_STRIP_MAX_L + 1)];  /* [w*(MAX_L+1)+h] = ln|Z_wh| */
    int32_t sign_z[(PNE_STRIP_MAX_L + 1) * (PNE_STRIP_MAX_L + 1)]; /* sign of Z_wh */
    double messages[4 * PNE_STRIP_MAX_CHI];  /* mR, mL, mD, mU (chi each, unit overlaps) */
    double eig_change;       /* largest last relative change of lambda over k */
    int32_t bp_sweeps;       /* BP iterations                                 */
    int32_t eig_iters;       /* largest power-iteration count over k          */
    pne_status status;       /* this tensor's status                          */
    int32_t iters[2 * (PNE_STRIP_MAX_L + 1)];  /* [o*(MAX_L+1)+k]: power iterations of
                                                  width k, o = 0 vertical, 1 horizontal */
} pne_strip_result;

pne_status pne_strip_expansion(pne_ctx *ctx, int32_t chi, int32_t n_tensors, const double *A, int32_t A_on_device,
                               const pne_strip_opts *opts, void *stream, pne_strip_result *out);

/* ---- dense contractions of blocked large-chi networks (tensor cores) ----- */

/* Batched dense product C[b] = A[b] B[b]^T on the device: A [M][K] (row stride
 * lda), B [N][K] (row stride ldb), C [M][N] (row stride ldc), set b at
 * offsets b * stride*.  All device pointers.
 *   PNE_TF32 / PNE_BF16: A, B, C FP32; the inputs rounded to TF32 (nearest,
 *     ties away) or BF16 (nearest-even) and multiplied on the 5th-generation
 *     tensor cores (tcgen05.mma, M = 128 tiles, N <= 256 per tile) with FP32
 *     accumulation in tensor memory: |error| <= (2 u_in + K 2^-24) sum_k |a b|
 *     to first order, u_in = 2^-11 (TF32) or 2^-8 (BF16).
 *   PNE_F64: A, B, C FP64, FP64 multiply-adds on the CUDA cores.
 * This is the primitive of pne_grid_contract.  Returns PNE_EINVAL on bad
 * sizes (batch 1..65535, M, N, K >= 1, lda, ldb >= K, ldc >= N) or PNE_F32,
 * PNE_ETIMEOUT if a tensor-core stage wait gave up (bounded at about 2 s).
 * Synchronises `stream`. */
pne_status pne_dense_gemm(pne_ctx *ctx, pne_dtype dtype, int32_t batch, int32_t M, int32_t N, int32_t K,
                          const void *A, int64_t lda, int64_t strideA, const void *B, int64_t ldb, int64_t strideB,
                          void *C, int64_t ldc, int64_t strideC, void *stream);

/* Exact contraction (Eq. A1) of a closed 2D grid network: the lattices the
 * paper coarse-grains into bond dimension chi = 16 or 64 (App. A) and
 * contracts exactly as the reference of its benchmarks and as the terms of
 * its expansions (Sec. III, Sec. IV.A).  Sites are an lx x ly grid, site id =
 * y * lx + x, and every bond joins grid neighbours (each neighbour pair by
 * exactly one bond, any dimension 1..4096); n_batch tensor sets, FP64 data on
 * the host or the device as for pne_build_partition.  The grid is contracted
 * row by row; absorbing a site is one dense product of the running tensor
 * (rows: its legs other than the site's up and left legs) with the site's
 * [down, right] x [up, left] matrix, scaled to a largest entry in [1, 2) by a
 * power of two each step (kept exactly in a log scale).
 *   dtype  PNE_F64 (FP64 products on the CUDA cores), PNE_TF32 or PNE_BF16
 *          (products on the tensor cores, FP32 running tensor and
 *          accumulation); PNE_F32 is rejected.
 *   out    [n_batch]: sign, log_abs, value of Z; err_bound = the first-order
 *          bound sum over sites of (2 u_in + K_site u_acc) on |error| / Z_abs,
 *          Z_abs the contraction of |T| (= |Z| for non-negative networks);
 *          n_terms = 1, c[0] = 1.
 * The running tensor holds at most prod of the open vertical bonds of a row
 * times two horizontal ones; PNE_EINVAL when the batch's running tensors would
 * exceed 64 GB, or on a network that is not such a grid.  On the tensor cores,
 * sites whose 16-byte operand units are contiguous are fed by TMA, with
 * clusters of 2 CTAs sharing the site matrix by multicast (the environment
 * variable PNE_TC_CLUSTER = 1, 2 or 4 sets the cluster size; results do not
 * depend on it).  Synchronises `stream`. */
pne_status pne_grid_contract(pne_ctx *ctx, const pne_network *net, int32_t lx, int32_t ly, pne_dtype dtype,
                             void *stream, pne_result *out);

/* The rank-r expansion of pne_rank_r_expand with every term contracted as a
 * 2D grid (the weighted network restricted to each term's index ranges,
 * contracted row by row as in pne_grid_contract): FP64 products on the CUDA
 * cores, or TF32 / BF16 products on the tensor cores with FP32 accumulation
 * -- the dense contractions of blocked large-chi networks (App. A, Sec. V).
 * The network of the weights must be an lx x ly grid (site id = y * lx + x).
 * Results as pne_rank_r_expand; err_bound adds, per term, the grid
 * contraction's bound times |term value| (exact for terms of non-negative
 * tensors, where the absolute contraction is the value).  PNE_F32 is rejected.
 * Synchronises `stream`. */
pne_status pne_rank_r_expand_grid(pne_ctx *ctx, const pne_weights *w, int32_t rank, int32_t form,
                                  int32_t n_partitions, const int32_t *partition_ptr, const int32_t *partition_bonds,
                                  int32_t lx, int32_t ly, pne_dtype dtype, void *stream, pne_result *out);

/* Recursive partitioning (Sec. IV.A) on the rank-r projectors of the weights:
 * the combinatorial form (Eq. A6) over the first-level partitions, in which
 * every sub-network with a connected component (sites joined by bonds not
 * cut by its partitions) too costly to contract -- on the lx x ly grid, both
 * sides of the component's bounding box above max_side (a strip w sites wide
 * carries w legs from row to row) -- is not contracted as it is but expanded
 * again by the combinatorial form over the second-level partitions that fit
 * inside its too-costly components (every bond of such a partition uncut
 * and joining two sites of one of them):
 *     Z(P^x) ~ sum_{y != 0} (-1)^{|y|+1} Z(P^x P^y),
 * the residues of both levels neglected.  A sub-network no second-level
 * partition fits is contracted as it is.  Every network is contracted as a
 * grid (pne_rank_r_expand_grid's contraction, dtype F64 / TF32 / BF16).
 * Results per tensor set as pne_rank_r_expand (c[k]: first-level subsets of
 * k partitions, each with its second-level sum); n_terms and
 * *n_contractions = networks contracted.  Limits: <= 16 first-level
 * partitions, <= 64 second-level partitions of which <= 16 fit any one
 * sub-network.  Synchronises `stream`. */
pne_status pne_recursive_expand_grid(pne_ctx *ctx, const pne_weights *w, int32_t rank, int32_t n_partitions,
                                     const int32_t *partition_ptr, const int32_t *partition_bonds,
                                     int32_t n_sub_partitions, const int32_t *sub_ptr, const int32_t *sub_bonds,
                                     int32_t max_side, int32_t lx, int32_t ly, pne_dtype dtype, void *stream,
                                     pne_result *out, uint64_t *n_contractions);

/* ---- belief propagation without device allocation ------------------------ */

/* The paper has no counterpart to this call.  It is for callers that must not
 * allocate device memory while they run: a host framework that has reserved
 * the device's memory for its own allocator and lends the library only fixed
 * buffers, or a latency-critical loop in which cudaMalloc / cudaFree (and the
 * device-wide synchronisation they can imply) are not allowed.  It runs the
 * same BP sweeps as pne_build_partition and returns the fixed-point messages,
 * but calls no cudaMalloc, cudaFree or allocating library routine: its working
 * memory (geometry tables, the second message buffer, convergence words) is a
 * file-scope device array of PNE_NOALLOC_SCRATCH_BYTES that every GPU which
 * loads the library holds until the process exits.
 *
 *   net        network as for pne_build_partition; net->data must be a device
 *              pointer (data_on_device != 0), n_batch tensor sets.  The
 *              geometry arrays are host arrays, copied with cudaMemcpyAsync.
 *   tol, max_iter  as in pne_partition_opts (defaults when <= 0).
 *   msg_out    device buffer [n_batch][site_ptr[n_sites]][8] doubles: for every
 *              leg slot (sites in order, each site's legs in ascending bond
 *              id) the outgoing fixed-point message, unit 2-norm, largest
 *              entry positive, zero-padded to 8 entries.
 *   iters_out, residual_out  host arrays [n_batch] (may be NULL): sweeps taken
 *              (0 = not converged) and the last sweep's largest change.
 * Returns PNE_EINVAL when the tables and buffers need more than
 * PNE_NOALLOC_SCRATCH_BYTES, checked on the host before any GPU work (or on
 * malformed input), PNE_ENOCONV, PNE_EDEGENERATE, PNE_ETIMEOUT or PNE_ECUDA as
 * pne_build_partition does.  Synchronises `stream` before it returns.  The
 * first call on a device looks up the array's device address (per device,
 * with that device current).  All calls share the one array and it keeps the
 * last call's contents (each call clears the words that must start at zero):
 * calls that overlap on the GPU (other streams, other host threads) race and
 * corrupt each other. */
#define PNE_NOALLOC_SCRATCH_BYTES (8u << 20)
pne_status pne_bp_messages_noalloc(const pne_network *net, double tol, int32_t max_iter, double *msg_out,
                                   int32_t *iters_out, double *residual_out, void *stream);

/* ---- measurement --------------------------------------------------------- */

/* Per-kernel timing with CUDA events recorded on the launching stream around
 * every kernel the library launches (no effect on results).  enable != 0
 * turns it on and clears the record; 0 turns it off.  enable == 2 also keeps
 * a timeline (pne_ctx_trace_read): the call then synchronises the device
 * once to fix the time origin. */
pne_status pne_ctx_profile(pne_ctx *ctx, int enable);

typedef struct {
    char name[32];        /* kernel family, e.g. "bp_sweep", "contract"       */
    int64_t launches;
    double total_ms;      /* sum of event-timed launch durations              */
} pne_profile_entry;

/* Waits for the recorded events, then writes up to max entries (sorted by
 * total time, largest first); returns the number of kernel families. */
int pne_ctx_profile_read(pne_ctx *ctx, pne_profile_entry *out, int max);

typedef struct {
    char name[32];        /* kernel family, or a host stretch of library code  */
    int32_t kind;         /* 0: kernel (event-timed on its stream), 1: host    */
    int32_t stream;       /* kernels: streams numbered by first appearance; -1 */
    double t0_ms, t1_ms;  /* since the origin set by pne_ctx_profile(ctx, 2)   */
} pne_trace_entry;

/* The timeline recorded since pne_ctx_profile(ctx, 2): waits for the recorded
 * events, writes up to max entries sorted by start time and returns how many
 * there are (at most 2^18 of each kind are kept).  Kernel times come from
 * events, host times from the steady clock; *host_origin_ms (may be NULL)
 * receives the steady-clock reading, in ms, taken when the origin event
 * completed, so that a caller's own monotonic timestamps can be placed on the
 * same axis.  The two clocks agree to within the event-completion latency. */
int pne_ctx_trace_read(pne_ctx *ctx, pne_trace_entry *out, int max, double *host_origin_ms);

/* Multiply-adds of every cluster's contraction plan, summed over clusters (one
 * tensor set): the algorithmic work of pne_contract_terms per tensor set.
 * LOOP mode.  Synchronises `stream`. */
pne_status pne_terms_work(pne_ctx *ctx, const pne_terms *t, void *stream, uint64_t *fma_per_set);

/* Sustained fused multiply-add throughput of this GPU's CUDA cores in FLOP/s
 * (2 per FMA) for PNE_F64 or PNE_F32, measured with an FMA-chain kernel; the
 * denominator of the ALU roofline.  Synchronises `stream`. */
pne_status pne_measure_fma_peak(pne_ctx *ctx, pne_dtype dtype, void *stream, double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif /* PNE_H */
