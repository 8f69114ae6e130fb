// Cluster and term enumeration on the GPU (integer work only).
//
// Clusters (Sec. III.A): connected sets C of closed bonds with |C| <= K.  In
// LOOP mode no site of C may have C-degree one (a dangling excitation, which
// vanishes at a BP fixed point).  Each connected set is generated exactly once
// from its smallest bond (the anchor) by a Redelmeier-style search: a node of
// the search tree is (S, U), S the current set and U the ordered list of
// candidate bonds still to try; taking U[i] gives the child
// (S + U[i], U[i+1..] ++ new), where `new` are the bonds at the site U[i]
// brings in (if any), larger than the anchor, whose other end is not yet in S.
// In LOOP mode a subtree is skipped when its set cannot be completed: more
// degree-one sites than 2 (K - |S|) (each further bond repairs at most two),
// or a degree-one site none of whose bonds is in the candidate list -- every
// bond that touches a site of S is either in S, in the list, or was already
// tried and is excluded from the subtree, and bonds found later join new
// sites only.
//
// Parallel schedule: the first levels of every anchor's tree are expanded
// level by level (one warp per node, one lane per candidate) into a node arena
// whose level bounds stay on the device, so the levels need no host round
// trip; each node of the last prefix level is then searched depth-first by one
// thread, unless the prefix already reaches size K - 1 and one more
// warp-parallel step ends it.  In LOOP mode the prefix stops at size K - 2:
// the bond that completes a cluster of size K joins two vertices the set
// already has, so a node of size K - 2 finds both remaining sizes in one
// warp-parallel step (each lane's child, then the child's closing bonds among
// the node's later candidates) and the far more numerous sets of size K - 1
// that cannot be closed are never stored; a child of size K - 2 is kept only
// if two more candidate bonds can still close it (closable2).  Every unit
// first counts what it emits per cluster size; an exclusive scan over (size,
// unit) gives each unit its output slots, and a second pass writes.  The
// output is grouped by size and deterministic.
//
// Terms (Eq. A4): a term is a set of pairwise vertex-disjoint clusters with
// total size <= K (the connected components of one P/Q string).  Tuples
// (i_1 < i_2 < ...) of cluster ids are built one length at a time, each
// extended by every larger id whose size fits and whose sites are disjoint.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstring>

#include "pne_internal.h"

namespace pne {

namespace {

constexpr int kPrefixMax = 8;     // deepest prefix level kept as explicit nodes
constexpr int kNodeU = 48;        // candidate-list capacity of a prefix node
constexpr int64_t kArenaFirst = 1 << 16;    // arena size of a first search (nodes), grown on demand
constexpr int64_t kNodeCap = 1 << 22;       // largest arena; beyond it the deepest level that fits is searched depth-first

constexpr int kNodeV = kPrefixMax + 2;   // vertex capacity of S plus one bond

// A node of the search tree: the set S (t bonds), its candidate list U, and the
// vertex multiset of S (vertices, C-degrees, count, degree-one count), so a
// child's multiset is its parent's plus the endpoints of one bond.
struct Node {
    int32_t S[kPrefixMax];
    int32_t U[kNodeU];
    int32_t nU;
    int32_t t;
    int32_t vn, vdang;
    int32_t vv[kNodeV], vd[kNodeV];
};

struct GeomView {
    const int32_t *bond_site;     // closed geometry [Mc][2]
    const int32_t *site_ptr, *site_bonds;
    const int2 *site_nbr;         // per leg: (bond, site at the other end)
};

__device__ __forceinline__ int2 bond_ends(const GeomView &g, int e)
{
    return __ldg(reinterpret_cast<const int2 *>(g.bond_site) + e);
}

struct Emit {
    int32_t *edges;               // [n][width]
    int32_t *verts;               // [n][vwidth]
    int32_t *size;                // [n]
    int width, vwidth;
};

// Vertex multiset of a bond set, with the number of degree-one vertices.
// Every loop runs over the fixed capacity NV with a guard on n, so after
// unrolling all indices are constants and the set lives in registers.
template <int NV>
struct VSet {
    int32_t v[NV];
    int32_t d[NV];
    int n = 0;
    int dang = 0;
    __device__ __forceinline__ bool has(int x) const {
        bool r = false;
#pragma unroll
        for (int i = 0; i < NV; ++i) r |= (i < n && v[i] == x);
        return r;
    }
    __device__ __forceinline__ void inc(int x) {
        int o = -1;
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (i < n && v[i] == x) { o = d[i]; d[i] = o + 1; }
        if (o < 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i)
                if (i == n) { v[i] = x; d[i] = 1; }
            ++n;
            o = 0;
        }
        if (o == 0) ++dang; else if (o == 1) --dang;
    }
    __device__ __forceinline__ void dec(int x) {       // x was the last vertex added if its degree drops to 0
        int o = 0;
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (i < n && v[i] == x) { o = d[i]; d[i] = o - 1; }
        if (o == 1) { --dang; --n; }
        else if (o == 2) ++dang;
    }
};

template <int NV>
__device__ __forceinline__ void load_vset(VSet<NV> &V, const Node &nd)
{
    V.n = nd.vn; V.dang = nd.vdang;
#pragma unroll
    for (int i = 0; i < (NV < kNodeV ? NV : kNodeV); ++i) { V.v[i] = nd.vv[i]; V.d[i] = nd.vd[i]; }
}

template <int NV>
__device__ __forceinline__ void store_vset(Node *nd, const VSet<NV> &V)
{
    nd->vn = V.n; nd->vdang = V.dang;
#pragma unroll
    for (int i = 0; i < (NV < kNodeV ? NV : kNodeV); ++i) { nd->vv[i] = V.v[i]; nd->vd[i] = V.d[i]; }
}

__device__ __forceinline__ bool valid_set(int mode, int dang) { return mode == PNE_MODE_ALL || dang == 0; }
__device__ __forceinline__ bool may_grow(int mode, int s, int K, int dang)
{
    return s < K && (mode == PNE_MODE_ALL || dang <= 2 * (K - s));
}

// every degree-one site of V has a bond among the candidates U[lo..hi)
template <int NV>
__device__ bool repairable(const VSet<NV> &V, const int32_t *UA, const int32_t *UB, int lo, int hi)
{
    if (V.dang == 0) return true;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i >= V.n) break;
        if (V.d[i] != 1) continue;
        const int x = V.v[i];
        bool found = false;
        for (int q = lo; q < hi; ++q)
            if (UA[q] == x || UB[q] == x) { found = true; break; }
        if (!found) return false;
    }
    return true;
}

template <int NV>
__device__ void write_cluster(const Emit &o, int64_t slot, const int32_t *S, int s, const VSet<NV> &V)
{
    int32_t *e = o.edges + slot * o.width;
    for (int i = 0; i < s; ++i) {            // insertion sort into the row
        int x = S[i], j = i;
        while (j > 0 && e[j - 1] > x) { e[j] = e[j - 1]; --j; }
        e[j] = x;
    }
    for (int i = s; i < o.width; ++i) e[i] = -1;
    int32_t *vv = o.verts + slot * o.vwidth;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        if (i >= V.n) break;
        int x = V.v[i], j = i;
        while (j > 0 && vv[j - 1] > x) { vv[j] = vv[j - 1]; --j; }
        vv[j] = x;
    }
    for (int i = V.n; i < o.vwidth; ++i) vv[i] = -1;
    o.size[slot] = s;
}

// Bonds at new vertex b (> anchor, other end not in V), appended to U.  The
// site's (bond, other end) pairs are loaded together first, so the walk costs
// two dependent loads, not two per bond.
template <int NV>
__device__ int append_new(const GeomView &g, int b, int e, int anchor, const VSet<NV> &V,
                          int32_t *U, int32_t *UA, int32_t *UB, int ne, int cap, int32_t *overflow)
{
    const int p0 = __ldg(g.site_ptr + b), p1 = __ldg(g.site_ptr + b + 1);
    int2 nb[kMaxDeg];
#pragma unroll
    for (int k = 0; k < kMaxDeg; ++k) nb[k] = (p0 + k < p1) ? __ldg(g.site_nbr + p0 + k) : make_int2(-1, -1);
#pragma unroll
    for (int k = 0; k < kMaxDeg; ++k) {
        const int f = nb[k].x, c = nb[k].y;
        if (p0 + k >= p1 || f == e || f <= anchor || V.has(c)) continue;
        if (ne >= cap) { atomicExch(overflow, 1); return ne; }
        U[ne] = f; UA[ne] = b; UB[ne] = c;
        ++ne;
    }
    return ne;
}

// ---------------------------------------------------------------- scan
// Exclusive prefix sums of int32 or int64 values into int64.  A tile is
// THREADS * kScanItems values scanned by one block: warp w owns kScanItems
// consecutive rows of 32 values, lane l column l, so loads and stores are
// coalesced; all loads of a tile are issued before the first shuffle, rows are
// scanned across lanes and chained through the last lane, and the warp totals
// are scanned by warp 0.  Small tables are scanned by one block walking the
// tiles with a running carry (one launch); larger ones by one block per tile,
// a scan of the tile totals, and an add pass.  `in` may alias `out`.
constexpr int kScanItems = 8;
constexpr int kScanTile = 1024 * kScanItems;
constexpr int64_t kOneBlockTiles = 4;

template <int THREADS, typename T>
__device__ __forceinline__ int64_t tile_scan(const T *in, int64_t *out, int64_t n, int64_t t0, int64_t carry,
                                             int64_t *wsum /* shared [THREADS / 32] */)
{
    constexpr int W = THREADS / 32;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t b = t0 + (int64_t)wid * (32 * kScanItems) + lane;
    int64_t v[kScanItems], x[kScanItems];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t at = b + 32 * k;
        v[k] = (at < n) ? (int64_t)in[at] : 0;
    }
    int64_t run = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int64_t y = v[k];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t z = __shfl_up_sync(0xffffffffu, y, off);
            if (lane >= off) y += z;
        }
        x[k] = run + y - v[k];
        run += __shfl_sync(0xffffffffu, y, 31);
    }
    if (lane == 0) wsum[wid] = run;
    __syncthreads();
    if (wid == 0) {
        int64_t ws = (lane < W) ? wsum[lane] : 0;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t z = __shfl_up_sync(0xffffffffu, ws, off);
            if (lane >= off) ws += z;
        }
        if (lane < W) wsum[lane] = ws;
    }
    __syncthreads();
    const int64_t before = carry + (wid > 0 ? wsum[wid - 1] : 0);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t at = b + 32 * k;
        if (at < n) out[at] = before + x[k];
    }
    const int64_t total = wsum[W - 1];
    __syncthreads();
    return total;
}

// exclusive scan of in[0, n) by the whole block, tile after tile; returns the total
template <int THREADS, typename T>
__device__ int64_t block_scan_range(const T *in, int64_t *out, int64_t n, int64_t *wsum)
{
    int64_t carry = 0;
    for (int64_t t0 = 0; t0 < n; t0 += THREADS * kScanItems) carry += tile_scan<THREADS>(in, out, n, t0, carry, wsum);
    return carry;
}

template <typename T>
__global__ void __launch_bounds__(1024) scan_one_block_kernel(const T *in, int64_t *out, int64_t n, int64_t *total)
{
    __shared__ int64_t wsum[32];
    const int64_t t = block_scan_range<1024>(in, out, n, wsum);
    if (threadIdx.x == 0) *total = t;
}

template <typename T>
__global__ void __launch_bounds__(1024) scan_tiles_kernel(const T *in, int64_t *out, int64_t n, int64_t *tile_sums)
{
    __shared__ int64_t wsum[32];
    const int64_t t = tile_scan<1024>(in, out, n, (int64_t)blockIdx.x * kScanTile, 0, wsum);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) scan_add_tiles_kernel(int64_t *out, int64_t n, const int64_t *tile_off)
{
    const int64_t add = tile_off[blockIdx.x];
    const int64_t b = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t at = b + 1024 * k;
        if (at < n) out[at] += add;
    }
}

// starts[r] = scanned[r * cols] (or the total at r == rows), one thread per row
__global__ void row_starts_kernel(const int64_t *scanned, int rows, int64_t cols, int64_t n, int64_t *starts,
                                  const int64_t *total)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > rows) return;
    const int64_t at = (int64_t)r * cols;
    starts[r] = (r == rows || at >= n) ? *total : scanned[at];
}


// ---------------------------------------------------------------- search arena
// Every prefix level lives in one node arena: level d (d = 1: the anchors,
// one node per bond) is nodes[lv[d-1], lv[d]).  Level sizes stay on the
// device, so the levels are expanded without a host round trip.  A level
// whose children would not fit stops the search (ctl->stop = d, ctl->need =
// the size it asked for) and every deeper level is left empty.  Count and
// slot tables are [K+1][cap], indexed by arena position.
struct SearchCtl {
    int32_t cand_overflow;        // a candidate list outgrew kNodeU
    int32_t stop;                 // first level whose children did not fit (0: none)
    int64_t need;                 // arena size that level asked for
};

struct Arena {
    Node *nodes;
    int64_t cap;
    int64_t *lv;                  // [kPrefixMax + 2] level boundaries
    int32_t *child_cnt;           // [cap] children per node
    int64_t *child_off;           // [cap] child offset within the node's chunk
    int64_t *chunk_tot;           // [grid] children per chunk, then their exclusive scan
    int32_t *counts;              // [K+1][cap] clusters emitted per (size, node)
    uint64_t *gmask, *emask;      // [cap] per node: candidates that make a child / an emitted cluster
    const int64_t *base;          // [K+1][cap] first output slot per (size, node)
    SearchCtl *ctl;
};

__global__ void arena_init_kernel(Arena a, int n_roots)
{
    if (threadIdx.x <= kPrefixMax + 1) a.lv[threadIdx.x] = threadIdx.x == 0 ? 0 : n_roots;
    if (threadIdx.x == 0) {
        a.ctl->cand_overflow = 0; a.ctl->stop = 0; a.ctl->need = 0;
    }
}

// ---------------------------------------------------------------- roots
__global__ void roots_kernel(GeomView g, int n_closed, int mode, Arena A, Emit out, int write)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < n_closed; a += gridDim.x * blockDim.x) {
        const int x0 = g.bond_site[2 * a], x1 = g.bond_site[2 * a + 1];
        if (!write) {
            Node nd;
            nd.S[0] = a; nd.t = 1;
            int n = 0;
            for (int p = g.site_ptr[x0]; p < g.site_ptr[x0 + 1]; ++p) {
                int f = g.site_bonds[p];
                if (f > a) { if (n < kNodeU) nd.U[n++] = f; else atomicExch(&A.ctl->cand_overflow, 1); }
            }
            for (int p = g.site_ptr[x1]; p < g.site_ptr[x1 + 1]; ++p) {
                int f = g.site_bonds[p];
                if (f <= a) continue;
                const int c = g.bond_site[2 * f] == x1 ? g.bond_site[2 * f + 1] : g.bond_site[2 * f];
                if (c == x0) continue;                 // parallel bond, already listed at x0
                if (n < kNodeU) nd.U[n++] = f; else atomicExch(&A.ctl->cand_overflow, 1);
            }
            nd.nU = n;
            VSet<kNodeV> V;
            V.inc(x0); V.inc(x1);
            store_vset(&nd, V);
            A.nodes[a] = nd;
            A.counts[1 * A.cap + a] = (mode == PNE_MODE_ALL) ? 1 : 0;
        } else if (mode == PNE_MODE_ALL) {
            VSet<2> V;
            V.inc(x0); V.inc(x1);
            int32_t S[1] = {a};
            write_cluster(out, A.base[1 * A.cap + a], S, 1, V);
        }
    }
}

// ---------------------------------------------------------------- prefix expansion
// One warp per node, one lane per candidate U[i] (two rounds when the list is
// longer than a warp).  Each lane forms S + U[i] on its own, so a node costs a
// few hundred instructions of latency instead of a serial walk over its list;
// ballots give every child and every emitted set its rank within the node, so
// the output order is the candidate order, as in the serial search.
// Block b takes the b-th contiguous chunk of the node range, its warps
// striding through it.
//   kCount:     children and emissions of level lo == hi; the block then scans
//               its chunk's child counts (offsets within the chunk, chunk total)
//   kEmitCount: emissions only (the last level)
//   kChildren:  write the children of level lo == hi, unless the search stopped
//   kEmit:      write the emitted clusters of levels lo..hi
//   kPairCount: the closing level of LOOP mode (nodes of size K - 2): sizes
//               K - 1 and K counted together, no nodes of size K - 1 made
//               (see pair_node)
enum ExpandPass { kCount = 0, kChildren = 1, kEmit = 2, kEmitCount = 3, kPairCount = 4 };
constexpr int kExpandWarps = 4;
constexpr int kMaxNew = kNodeU / (kPrefixMax + 1);   // new candidates per step (site degree - 1)
constexpr int kNodeWords = (int)(sizeof(Node) / 4);

// Node word offsets (the children are written word by word) and the staging
// record of a growing lane: new-candidate count, new candidates, then the
// bond's end indices in the node's vertex list, the vertex it brings in and
// the child's degree-one count.
constexpr int kOffNU = (int)(offsetof(Node, nU) / 4);
constexpr int kOffT = (int)(offsetof(Node, t) / 4);
constexpr int kOffVN = (int)(offsetof(Node, vn) / 4);
constexpr int kStageWords = 1 + kMaxNew + 4;
static_assert(offsetof(Node, vdang) / 4 == kOffVN + 1 && offsetof(Node, vv) / 4 == kOffVN + 2 &&
              offsetof(Node, vd) / 4 == kOffVN + 2 + kNodeV && sizeof(Node) / 4 == kOffVN + 2 + 2 * kNodeV,
              "node layout");
static_assert(kNodeV <= 32 && kNodeU <= 64, "vertex and candidate masks");

// Per-node tables of one warp, in shared memory.  Every candidate U[q] touches
// the node's vertex set; ia[q] and ib[q] are the indices of its two ends in
// the node's vertex list (-1: not in it), so the child S + U[q] is described
// relative to the node: the bond raises the degrees of ia and ib, and brings
// in the vertex outside(q) when one end is missing.
struct NodeTabs {
    int32_t *UA, *UB;         // ends of U[q]
    int32_t *ia, *ib;         // their indices in the node's vertex list, -1: outside
    uint64_t *tmask;          // [vn] candidates at vertex k (counting pass)
    int32_t *tw;              // last other candidate with the same outside end (-1: none)
    __device__ __forceinline__ int outside(int q) const { return ia[q] < 0 ? UA[q] : (ib[q] < 0 ? UB[q] : -1); }
};

// The child S + U[i] relative to the node: its degree-one vertices are the
// node's degree-one vertices the bond does not touch (mask over the vertex
// list) plus the vertex b it brings in.
struct Child {
    int ia, ib, b;
    uint32_t dmask;           // degree-one vertices of the node still at degree one
    int dang;                 // the child's degree-one count
};

__device__ __forceinline__ Child make_child(const NodeTabs &T, int i, uint32_t node_dmask)
{
    Child c;
    c.ia = T.ia[i]; c.ib = T.ib[i];
    c.b = c.ia < 0 ? T.UA[i] : (c.ib < 0 ? T.UB[i] : -1);
    c.dmask = node_dmask & ~((c.ia >= 0 ? 1u << c.ia : 0u) | (c.ib >= 0 ? 1u << c.ib : 0u));
    c.dang = __popc(c.dmask) + (c.b >= 0 ? 1 : 0);
    return c;
}

// Bonds at the new vertex b (> anchor, not e, other end outside the node's
// vertex list vv[0, vn)): the child's new candidates, in the site's leg order.
// The site's (bond, other end) pairs are loaded together, so the walk costs
// two dependent loads.
__device__ __forceinline__ int new_candidates(const GeomView &g, int b, int e, int anchor, const int32_t *vv, int vn,
                                              int32_t *NU, int32_t *NB, int32_t *overflow)
{
    const int p0 = __ldg(g.site_ptr + b), p1 = __ldg(g.site_ptr + b + 1);
    int2 nb[kMaxDeg];
#pragma unroll
    for (int k = 0; k < kMaxDeg; ++k) nb[k] = (p0 + k < p1) ? __ldg(g.site_nbr + p0 + k) : make_int2(-1, -1);
    int ne = 0;
#pragma unroll
    for (int k = 0; k < kMaxDeg; ++k) {
        const int f = nb[k].x, c = nb[k].y;
        if (p0 + k >= p1 || f == e || f <= anchor) continue;
        bool in = false;
        for (int j = 0; j < vn; ++j) in |= vv[j] == c;
        if (in) continue;
        if (ne >= kMaxNew) { atomicExch(overflow, 1); break; }
        NU[ne] = f; NB[ne] = c;
        ++ne;
    }
    return ne;
}

// Every degree-one vertex of the child can still be repaired inside its
// subtree: a vertex of the node iff some candidate after i touches it; the
// vertex b iff it has new candidates or a later candidate touches it.
__device__ __forceinline__ bool repairable_child(const NodeTabs &T, const Child &c, int i, int nn, int nU)
{
    for (uint32_t m = c.dmask; m; m &= m - 1) {
        const int k = __ffs(m) - 1;
        if ((T.tmask[k] >> (i + 1)) == 0) return false;
    }
    if (c.b >= 0 && nn == 0) {
        bool found = false;
        for (int q = i + 1; q < nU && !found; ++q) found = T.outside(q) == c.b;
        if (!found) return false;
    }
    return true;
}

// Can the child S + U[i] (size K - 2, LOOP mode) still be closed with the two
// bonds left?  Both must come from the child's candidate list (a bond of a
// new candidate list leads to a vertex outside the set and leaves it with
// degree one).  So every degree-one vertex v of the child needs, among those
// candidates, a bond from v to a vertex of the child (cost 1) or two bonds
// through one vertex w outside the child, one of them at v (cost 2).  Charging
// each degree-one vertex to the bond ends that serve it (a bond has two ends,
// a path through w four, serving at most two such vertices) shows that the
// costs of a closable child sum to at most 4.  The candidates of the child
// are U[j], j > i, and its new candidates (b, nb[k]), k < nn.
__device__ bool closable2(const NodeTabs &T, const Child &c, int i, int nn, const int32_t *nb, int nU)
{
    if (c.dang > 4) return false;
    const uint64_t after = ~0ull << (i + 1);
    auto in_nb = [&](int w) {
        bool f = false;
        for (int k = 0; k < nn; ++k) f |= nb[k] == w;
        return f;
    };
    int sum = 0;
    for (uint32_t dm = c.dmask; dm; dm &= dm - 1) {
        const int k = __ffs(dm) - 1;
        uint64_t m = T.tmask[k] & after;
        int cost = 3;
        while (m) {
            const int q = __ffsll((long long)m) - 1;
            m &= m - 1;
            const int w = T.outside(q);
            if (w < 0 || w == c.b) { cost = 1; break; }            // a bond to a vertex of the child
            if (T.tw[q] > i || (c.b >= 0 && in_nb(w))) cost = 2;   // a second bond at w: later, or new from b
        }
        if (cost > 2) return false;
        sum += cost;
    }
    if (c.b >= 0) {
        if (T.tw[i] > i) {
            sum += 1;            // a later candidate joins b to the node's vertex set
        } else {
            // a path b - x - y through one of b's new far ends x: a later
            // candidate with outside end x, or a second new bond to x
            if (sum + 2 > 4) return false;
            bool ok = false;
            for (int k = 0; k < nn && !ok; ++k)
                for (int k2 = k + 1; k2 < nn; ++k2) ok |= nb[k] == nb[k2];
            for (int q = i + 1; q < nU && !ok; ++q) ok = in_nb(T.outside(q));
            if (!ok) return false;
            sum += 2;
        }
    }
    return sum <= 4;
}

// Sorts N values in registers (odd-even transposition; every index constant).
template <int N>
__device__ __forceinline__ void sort_regs(int32_t (&x)[N])
{
#pragma unroll
    for (int r = 0; r < N; ++r)
#pragma unroll
        for (int j = r & 1; j + 1 < N; j += 2) {
            const int lo = min(x[j], x[j + 1]), hi = max(x[j], x[j + 1]);
            x[j] = lo; x[j + 1] = hi;
        }
}

// Writes the cluster S + e1 (+ e2 when >= 0) of a node: bonds and vertices
// (the node's list plus b when >= 0) sorted ascending, rows padded with -1.
__device__ void write_child_cluster(const Emit &o, int64_t slot, const Node &nd, int e1, int e2, int b)
{
    constexpr int NS = kPrefixMax + 2, NVx = kNodeV + 1;
    const int t = nd.t, vn = nd.vn;
    int32_t sv[NS], vv[NVx];
#pragma unroll
    for (int q = 0; q < kPrefixMax; ++q) sv[q] = q < t ? nd.S[q] : INT_MAX;
    sv[kPrefixMax] = e1;
    sv[kPrefixMax + 1] = e2 >= 0 ? e2 : INT_MAX;
#pragma unroll
    for (int q = 0; q < kNodeV; ++q) vv[q] = q < vn ? nd.vv[q] : INT_MAX;
    vv[kNodeV] = b >= 0 ? b : INT_MAX;
    sort_regs(sv);
    sort_regs(vv);
    const int s = t + 1 + (e2 >= 0 ? 1 : 0), n = vn + (b >= 0 ? 1 : 0);
    int32_t *er = o.edges + slot * o.width;
#pragma unroll
    for (int q = 0; q < NS; ++q)
        if (q < o.width) er[q] = q < s ? sv[q] : -1;
    for (int q = NS; q < o.width; ++q) er[q] = -1;
    int32_t *vr = o.verts + slot * o.vwidth;
#pragma unroll
    for (int q = 0; q < NVx; ++q)
        if (q < o.vwidth) vr[q] = q < n ? vv[q] : -1;
    for (int q = NVx; q < o.vwidth; ++q) vr[q] = -1;
    o.size[slot] = s;
}

// A node of size K - 2 in LOOP mode, both remaining levels at once.  Its child
// S + U[i] (size K - 1) is a cluster iff it has no degree-one vertex; a
// cluster of size K below that child is S + U[i] + U[j] with a bond U[j] of
// the child's candidate list that removes every degree-one vertex without
// adding one: both ends of U[j] already belong to the child, so U[j] is not
// one of the child's new candidates (those lead off the child's vertex set)
// and is a later candidate U[j], j > i, of this node.  It closes the child
// iff its ends include every degree-one vertex of the child (there are at
// most two).  The sizes K - 1 and K come out in the order of the level-by-
// level search: child by child, and per child in candidate order.
//   counting (kPairCount): per node the size K - 1 and size K counts, the
//     lanes with an emitted child (emask) and with a closing bond (gmask)
//   writing (kEmit): both sizes, from the slots of the (size, node) scan
// `want` is the lane mask of the writing pass.
template <int PASS>
__device__ void pair_node(const Arena &A, const Node &nd, int64_t u, const NodeTabs &T, uint32_t node_dmask,
                          uint64_t want, const Emit &out)
{
    constexpr int pass = PASS;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int nU = nd.nU, t = nd.t;
    int n_emit = 0, n_pair = 0;
    uint64_t emask = 0, pmask = 0;
    const int64_t ebase = (pass == kEmit) ? A.base[(int64_t)(t + 1) * A.cap + u] : 0;
    const int64_t pbase = (pass == kEmit) ? A.base[(int64_t)(t + 2) * A.cap + u] : 0;
    for (int i0 = 0; i0 < nU; i0 += 32) {
        const int i = i0 + lane;
        bool emit = false;
        int np = 0, d0 = -1, d1 = -1;
        Child c{-1, -1, -1, 0u, 0};
        const bool mine = i < nU && ((want >> i) & 1);
        if (mine) {
            c = make_child(T, i, node_dmask);
            emit = c.dang == 0;
            if (c.dang <= 2) {
                for (uint32_t m = c.dmask; m; m &= m - 1) {
                    const int v = nd.vv[__ffs(m) - 1];
                    if (d0 < 0) d0 = v; else d1 = v;
                }
                if (c.b >= 0) { if (d0 < 0) d0 = c.b; else d1 = c.b; }
                for (int j = i + 1; j < nU; ++j) {
                    const int oj = T.outside(j);
                    if (oj != -1 && oj != c.b) continue;
                    const int x = T.UA[j], y = T.UB[j];
                    if ((d0 >= 0 && d0 != x && d0 != y) || (d1 >= 0 && d1 != x && d1 != y)) continue;
                    ++np;
                }
            }
        }
        const unsigned em = __ballot_sync(0xffffffffu, emit), pm = __ballot_sync(0xffffffffu, np > 0);
        emask |= (uint64_t)em << i0;
        pmask |= (uint64_t)pm << i0;
        int incl = np;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += z;
        }
        if (pass == kEmit && mine) {
            const int ei = nd.U[i];
            if (emit) write_child_cluster(out, ebase + n_emit + __popc(em & lt), nd, ei, -1, c.b);
            int64_t slot = pbase + n_pair + (incl - np);
            if (np > 0)
                for (int j = i + 1; j < nU; ++j) {
                    const int oj = T.outside(j);
                    if (oj != -1 && oj != c.b) continue;
                    const int x = T.UA[j], y = T.UB[j];
                    if ((d0 >= 0 && d0 != x && d0 != y) || (d1 >= 0 && d1 != x && d1 != y)) continue;
                    write_child_cluster(out, slot++, nd, ei, nd.U[j], c.b);
                }
        }
        n_emit += __popc(em);
        n_pair += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (pass == kPairCount && lane == 0) {
        A.counts[(int64_t)(t + 1) * A.cap + u] = n_emit;
        A.counts[(int64_t)(t + 2) * A.cap + u] = n_pair;
        A.emask[u] = emask;
        A.gmask[u] = pmask;
    }
}

// The block's chunk of the node range [r0, r1).  kChildren writes the
// children from arena slot next + cbase_chunk on (cbase_chunk: the children of
// the chunks before this one).
// With FUSE, nodes of size K - 2 (LOOP mode) are closing nodes (pair_node).
// One instance per pass keeps each kernel's code small enough for the
// instruction cache.
template <int PASS, bool FUSE>
__device__ void expand_chunk(const GeomView &g, const Arena &A, int64_t r0, int64_t r1, int K, int mode,
                             const Emit &out, int64_t next, int64_t cbase_chunk)
{
    constexpr int pass = PASS;
    constexpr bool fuse = FUSE;
    __shared__ Node sh_node[kExpandWarps];
    __shared__ int32_t sh_a[kExpandWarps][kNodeU], sh_b[kExpandWarps][kNodeU];
    __shared__ int32_t sh_ia[kExpandWarps][kNodeU], sh_ib[kExpandWarps][kNodeU];
    __shared__ uint64_t sh_tmask[kExpandWarps][kNodeV];
    __shared__ int32_t sh_tw[kExpandWarps][kNodeU];
    __shared__ int32_t sh_stage[kExpandWarps][32 * kStageWords];
    __shared__ int64_t wsum[kExpandWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    Node &nd = sh_node[w];
    const NodeTabs T{sh_a[w], sh_b[w], sh_ia[w], sh_ib[w], sh_tmask[w], sh_tw[w]};
    int32_t *stage = sh_stage[w];
    // the counting and children passes take contiguous chunks (the child
    // offsets are scanned per chunk); the others stride over the whole range,
    // so the costly nodes of the deepest level spread over every block
    constexpr bool chunked = pass == kCount || pass == kChildren;
    const int64_t chunk = (r1 - r0 + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = chunked ? r0 + (int64_t)blockIdx.x * chunk : r0 + (int64_t)blockIdx.x * kExpandWarps;
    const int64_t c1 = chunked ? (c0 + chunk < r1 ? c0 + chunk : r1) : r1;
    const int64_t ustep = chunked ? kExpandWarps : (int64_t)gridDim.x * kExpandWarps;
    for (int64_t u = c0 + w; u < c1; u += ustep) {
        // the writing passes replay the counting pass's decisions: nodes that
        // make nothing are skipped, and only the lanes with a set bit work
        uint64_t want = ~0ull;
        if (pass == kChildren) want = __ldcg(reinterpret_cast<const unsigned long long *>(A.gmask + u));
        else if (pass == kEmit) want = __ldcg(reinterpret_cast<const unsigned long long *>(A.emask + u));
        if (pass == kEmit && fuse && __ldcg(&A.nodes[u].t) == K - 2)   // a closing node: lanes with a closing bond too
            want |= __ldcg(reinterpret_cast<const unsigned long long *>(A.gmask + u));
        if (want == 0) continue;
        // L2 loads: these nodes were written by other blocks
        const int32_t *src = reinterpret_cast<const int32_t *>(A.nodes + u);
        for (int q = lane; q < kNodeWords; q += 32) reinterpret_cast<int32_t *>(&nd)[q] = __ldcg(src + q);
        __syncwarp();
        const int nU = nd.nU, t = nd.t, anchor = nd.S[0], vn = nd.vn;
        for (int q = lane; q < nU; q += 32) {
            const int2 ab = bond_ends(g, nd.U[q]);
            int ia = -1, ib = -1;
            for (int k = 0; k < vn; ++k) {
                const int x = nd.vv[k];
                ia = x == ab.x ? k : ia;
                ib = x == ab.y ? k : ib;
            }
            T.UA[q] = ab.x; T.UB[q] = ab.y; T.ia[q] = ia; T.ib[q] = ib;
        }
        const uint32_t dmask = __ballot_sync(0xffffffffu, lane < vn && nd.vd[lane] == 1);
        __syncwarp();
        if (fuse && t == K - 2) {
            pair_node<PASS>(A, nd, u, T, dmask, want, out);
            __syncwarp();
            continue;
        }
        const bool closing_children = pass == kCount && fuse && t + 1 == K - 2;
        if (pass == kCount) {
            // the candidates at each vertex of the node
            for (int k = 0; k < vn; ++k) {
                const unsigned m0 = __ballot_sync(0xffffffffu, lane < nU && (T.ia[lane] == k || T.ib[lane] == k));
                const unsigned m1 = __ballot_sync(0xffffffffu, lane + 32 < nU && (T.ia[lane + 32] == k || T.ib[lane + 32] == k));
                if (lane == 0) T.tmask[k] = (uint64_t)m0 | ((uint64_t)m1 << 32);
            }
            if (closing_children) {
                // children are closing nodes: the twin table of closable2
                // (lanes of one round with the same outside end found by a
                // match; the other round, when there is one, walked)
                for (int i0 = 0; i0 < nU; i0 += 32) {
                    const int q = i0 + lane;
                    const int o = q < nU ? T.outside(q) : -2 - lane;
                    const unsigned m = __match_any_sync(0xffffffffu, o) & ~(1u << lane);
                    int lw = -1;
                    if (o >= 0) {
                        if (m) lw = i0 + 31 - __clz(m);
                        if (i0 == 0)
                            for (int f = 32; f < nU; ++f) lw = T.outside(f) == o ? f : lw;
                        else if (!m)
                            for (int f = 0; f < 32; ++f) lw = T.outside(f) == o ? f : lw;
                    }
                    if (q < nU) T.tw[q] = lw;
                }
            }
            __syncwarp();
        }
        int n_child = 0, n_emit = 0;
        const int64_t cbase = (pass == kChildren) ? next + cbase_chunk + __ldcg(A.child_off + u) : 0;
        const int64_t ebase = (pass == kEmit) ? A.base[(int64_t)(t + 1) * A.cap + u] : 0;
        uint64_t gmask = 0, emask = 0;
        for (int i0 = 0; i0 < nU; i0 += 32) {
            const int i = i0 + lane;
            bool emit = false, grow = false;
            int32_t NU[kMaxNew], NB[kMaxNew];
            int nn = 0;
            Child c{-1, -1, -1, 0u, 0};
            const bool mine = i < nU && ((want >> i) & 1);
            if (mine) {
                c = make_child(T, i, dmask);
                const int e = nd.U[i];
                if (pass == kChildren) {
                    // decided by the counting pass; only the new candidates are rebuilt
                    grow = true;
                    if (c.b >= 0) nn = new_candidates(g, c.b, e, anchor, nd.vv, vn, NU, NB, &A.ctl->cand_overflow);
                } else if (pass == kEmit) {
                    emit = true;
                } else {
                    emit = valid_set(mode, c.dang);
                    if (pass == kCount && may_grow(mode, t + 1, K, c.dang)) {
                        if (c.b >= 0) nn = new_candidates(g, c.b, e, anchor, nd.vv, vn, NU, NB, &A.ctl->cand_overflow);
                        grow = mode == PNE_MODE_ALL || repairable_child(T, c, i, nn, nU);
                        if (closing_children && grow) grow = closable2(T, c, i, nn, NB, nU);
                    }
                }
            }
            const unsigned gm = __ballot_sync(0xffffffffu, grow), em = __ballot_sync(0xffffffffu, emit);
            gmask |= (uint64_t)gm << i0;
            emask |= (uint64_t)em << i0;
            if (pass == kChildren && gm) {
                // each growing lane stages what its child adds; then the warp
                // writes the children one after another, 32 words per store
                if (grow) {
                    int32_t *st = stage + lane * kStageWords;
                    st[0] = nn;
                    for (int q = 0; q < nn; ++q) st[1 + q] = NU[q];
                    st[1 + kMaxNew] = c.ia;
                    st[2 + kMaxNew] = c.ib;
                    st[3 + kMaxNew] = c.b;
                    st[4 + kMaxNew] = c.dang;
                }
                __syncwarp();
                unsigned rem = gm;
                for (int r = 0; rem; ++r) {
                    const int o = __ffs(rem) - 1;
                    rem &= rem - 1;
                    const int io = i0 + o;
                    const int32_t *so = stage + o * kStageWords;
                    const int m0 = nU - io - 1, nno = so[0];
                    const int cia = so[1 + kMaxNew], cib = so[2 + kMaxNew], cb = so[3 + kMaxNew];
                    int32_t *cw = reinterpret_cast<int32_t *>(A.nodes + cbase + n_child + r);
                    for (int q = lane; q < kNodeWords; q += 32) {
                        int32_t val;
                        if (q < kPrefixMax) {
                            val = q < t ? nd.S[q] : (q == t ? nd.U[io] : 0);
                        } else if (q < kPrefixMax + kNodeU) {
                            const int idx = q - kPrefixMax;
                            val = idx < m0 ? nd.U[io + 1 + idx] : (idx - m0 < nno ? so[1 + idx - m0] : 0);
                        } else if (q == kOffNU) {
                            val = m0 + nno < kNodeU ? m0 + nno : kNodeU;
                        } else if (q == kOffT) {
                            val = t + 1;
                        } else if (q == kOffVN) {
                            val = vn + (cb >= 0 ? 1 : 0);
                        } else if (q == kOffVN + 1) {
                            val = so[4 + kMaxNew];
                        } else if (q < kOffVN + 2 + kNodeV) {
                            const int j = q - (kOffVN + 2);                       // vertex list: the node's, then b
                            val = j < vn ? nd.vv[j] : (j == vn && cb >= 0 ? cb : 0);
                        } else {
                            const int j = q - (kOffVN + 2 + kNodeV);              // degrees
                            val = j < vn ? nd.vd[j] + (j == cia ? 1 : 0) + (j == cib ? 1 : 0)
                                         : (j == vn && cb >= 0 ? 1 : 0);
                        }
                        cw[q] = val;
                    }
                    if (lane == 0 && m0 + nno > kNodeU) atomicExch(&A.ctl->cand_overflow, 1);
                }
                __syncwarp();
            }
            if (pass == kEmit && emit)
                write_child_cluster(out, ebase + n_emit + __popc(em & lt), nd, nd.U[i], -1, c.b);
            n_child += __popc(gm);
            n_emit += __popc(em);
        }
        if ((pass == kCount || pass == kEmitCount) && lane == 0) {
            A.counts[(int64_t)(t + 1) * A.cap + u] = n_emit;
            A.emask[u] = emask;
            if (pass == kCount) { A.child_cnt[u] = n_child; A.gmask[u] = gmask; }
        }
        __syncwarp();
    }
    if (pass == kCount) {
        __syncthreads();
        const int64_t len = c1 > c0 ? c1 - c0 : 0;
        const int64_t tot = block_scan_range<32 * kExpandWarps>(A.child_cnt + c0, A.child_off + c0, len, wsum);
        if (threadIdx.x == 0) A.chunk_tot[blockIdx.x] = tot;
    }
    __syncthreads();                                   // the shared node buffers are reused by the caller
}

// kCount / kEmitCount / kPairCount of level lo == hi, or kEmit over levels lo..hi
template <int PASS, bool FUSE>
__global__ void __launch_bounds__(32 * kExpandWarps, 6)
expand_kernel(GeomView g, Arena A, int lo_level, int hi_level, int K, int mode, Emit out)
{
    expand_chunk<PASS, FUSE>(g, A, A.lv[lo_level - 1], A.lv[hi_level], K, mode, out, 0, 0);
}

// One level step is two ordinary launches (no grid barrier, so the search can
// share the GPU with other streams' work): expand_kernel(kCount) for level d,
// then this kernel, which derives each block's child offset and the level's
// size from the chunk totals, places level d + 1 (or records the stop, block 0)
// and writes the children.  Every block reaches the same decision.
__global__ void __launch_bounds__(32 * kExpandWarps) expand_children_kernel(GeomView g, Arena A, int d, int K, int mode)
{
    __shared__ int64_t red[2][32 * kExpandWarps];
    Emit none{nullptr, nullptr, nullptr, 0, 0};
    if (A.ctl->stop != 0) return;                      // an earlier level stopped the search
    const int64_t lo = A.lv[d - 1], hi = A.lv[d];
    int64_t before = 0, total = 0;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += blockDim.x) {
        const int64_t c = A.chunk_tot[q];
        total += c;
        if (q < (int)blockIdx.x) before += c;
    }
    red[0][threadIdx.x] = before; red[1][threadIdx.x] = total;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
        }
        __syncthreads();
    }
    before = red[0][0]; total = red[1][0];
    __syncthreads();
    const bool fits = hi + total <= A.cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int e = d + 1; e <= kPrefixMax + 1; ++e) A.lv[e] = fits ? hi + total : hi;
        if (!fits) { A.ctl->stop = d; A.ctl->need = hi + total; }
    }
    if (!fits) return;
    expand_chunk<kChildren, false>(g, A, lo, hi, K, mode, none, hi, before);
}

// ---------------------------------------------------------------- depth-first tasks
// One thread searches the whole subtree below one node of `level`; counts go
// to rows t0 + 1 .. K of its arena column, writes to the slots those rows give.
template <int KMAX, int UMAX>
__global__ void __launch_bounds__(128) dfs_kernel(GeomView g, Arena A, int level, int K, int mode, int write, Emit out)
{
    const int64_t r0 = A.lv[level - 1], r1 = A.lv[level];
    for (int64_t u = r0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < r1;
         u += (int64_t)gridDim.x * blockDim.x) {
        const Node &nd = A.nodes[u];
        const int t0 = nd.t, anchor = nd.S[0];
        VSet<KMAX + 1> V;
        load_vset(V, nd);
        int32_t S[KMAX];
        int s = t0;
        for (int i = 0; i < t0; ++i) S[i] = nd.S[i];
        int32_t U[UMAX], UA[UMAX], UB[UMAX];
        for (int i = 0; i < nd.nU; ++i) {
            U[i] = nd.U[i];
            const int2 ab = bond_ends(g, U[i]);
            UA[i] = ab.x; UB[i] = ab.y;
        }
        int32_t pos[KMAX], end[KMAX];
        int32_t cnt[KMAX + 1];
        int64_t slot[KMAX + 1];
        for (int q = 0; q <= KMAX; ++q) {
            cnt[q] = 0;
            slot[q] = (write && q <= K) ? A.base[(int64_t)q * A.cap + u] : 0;
        }
        int lvl = 0;
        pos[0] = 0; end[0] = nd.nU;
        for (;;) {
            if (pos[lvl] >= end[lvl]) {
                if (lvl == 0) break;
                --lvl;
                const int e = S[--s];
                const int2 ab = bond_ends(g, e);
                V.dec(ab.y); V.dec(ab.x);
                ++pos[lvl];
                continue;
            }
            const int e = U[pos[lvl]];
            const int2 ab = bond_ends(g, e);
            const int a0 = ab.x, a1 = ab.y;
            const int b = !V.has(a0) ? a0 : (!V.has(a1) ? a1 : -1);
            V.inc(a0); V.inc(a1);
            S[s++] = e;
            if (valid_set(mode, V.dang)) {
                if (write) write_cluster(out, slot[s]++, S, s, V);
                else ++cnt[s];
            }
            if (may_grow(mode, s, K, V.dang)) {
                int ne = end[lvl];
                if (b >= 0) ne = append_new(g, b, e, anchor, V, U, UA, UB, ne, UMAX, &A.ctl->cand_overflow);
                if (mode == PNE_MODE_ALL || repairable(V, UA, UB, pos[lvl] + 1, ne)) {
                    ++lvl;
                    pos[lvl] = pos[lvl - 1] + 1;
                    end[lvl] = ne;
                    continue;
                }
            }
            --s;
            V.dec(a1); V.dec(a0);
            ++pos[lvl];
        }
        if (!write)
            for (int q = t0 + 1; q <= K; ++q) A.counts[(int64_t)q * A.cap + u] = cnt[q];
    }
}

// ---------------------------------------------------------------- tuples
struct TupleParams {
    const int32_t *verts;     // [n][vwidth] sorted, -1 pad
    const int32_t *size;      // [n]
    int vwidth, K, m;         // m: length of the input tuples
    const int32_t *in;        // [n_in][m] input tuples (m == 1: the anchors are cluster ids)
    const int32_t *in_order;  // [n_in] order of each input tuple
    int64_t n_in;
    const int64_t *size_end;  // [K+2]: first cluster index with size > s  (size_end[s])
    const int64_t *unit_off;  // [n_in + 1] chunk offsets
    int64_t n_units;
    int32_t *counts;          // [K+1][n_units]
    const int64_t *base;      // [K+1][n_units]
    int32_t *out;             // [n_out][m+1]
    int32_t *out_order;
};

constexpr int kTupleChunk = 128;

__device__ __forceinline__ bool disjoint_sorted(const int32_t *a, const int32_t *b, int w)
{
    // both sorted ascending, -1 padded at the end
    int i = 0, j = 0;
    while (i < w && j < w && a[i] >= 0 && b[j] >= 0) {
        if (a[i] == b[j]) return false;
        if (a[i] < b[j]) ++i; else ++j;
    }
    return true;
}

__global__ void tuple_chunks_kernel(TupleParams p, int64_t *n_chunks)
{
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < p.n_in;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *tp = p.in + t * p.m;
        const int last = tp[p.m - 1];
        const int o = p.in_order[t];
        int64_t lo = (int64_t)last + 1, hi = (o < p.K) ? p.size_end[p.K - o] : lo;
        int64_t nc = hi > lo ? (hi - lo + kTupleChunk - 1) / kTupleChunk : 0;
        n_chunks[t] = nc;
    }
}

// One warp per unit (an input tuple and a chunk of up to kTupleChunk candidate
// clusters), one lane per candidate.  A candidate's order is the tuple's order
// plus its size; lanes with the same order are ranked by __match_any_sync, and
// the per-order running counts of the warp sit in shared memory, so the output
// keeps candidate order within every (order, unit) slot range.
constexpr int kTupleWarps = 4;

__global__ void __launch_bounds__(32 * kTupleWarps) tuple_kernel(TupleParams p, int write)
{
    extern __shared__ int32_t tsh[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const int tv_words = p.m * p.vwidth;
    int32_t *tv = tsh + w * (tv_words + kMaxOrder + 1);     // the tuple's sorted vertex lists
    int32_t *cnt = tv + tv_words;                            // [K+1] running counts per order
    for (int64_t u = (int64_t)blockIdx.x * kTupleWarps + w; u < p.n_units; u += (int64_t)gridDim.x * kTupleWarps) {
        // locate the input tuple of this unit (binary search in unit_off)
        int64_t lo = 0, hi = p.n_in;
        while (hi - lo > 1) {
            int64_t mid = (lo + hi) / 2;
            if (p.unit_off[mid] <= u) lo = mid; else hi = mid;
        }
        const int64_t t = lo;
        const int64_t chunk = u - p.unit_off[t];
        const int32_t *tp = p.in + t * p.m;
        const int last = tp[p.m - 1];
        const int o = p.in_order[t];
        for (int q = lane; q < tv_words; q += 32) tv[q] = p.verts[(int64_t)tp[q / p.vwidth] * p.vwidth + q % p.vwidth];
        for (int q = lane; q <= p.K; q += 32) cnt[q] = 0;
        __syncwarp();
        const int64_t j0 = (int64_t)last + 1 + chunk * kTupleChunk;
        int64_t j1 = p.size_end[p.K - o];
        if (j1 > j0 + kTupleChunk) j1 = j0 + kTupleChunk;
        for (int64_t jb = j0; jb < j1; jb += 32) {
            const int64_t j = jb + lane;
            bool ok = j < j1;
            int ord = -1;
            if (ok) {
                const int32_t *vj = p.verts + j * p.vwidth;
                for (int q = 0; q < p.m && ok; ++q) ok = disjoint_sorted(tv + q * p.vwidth, vj, p.vwidth);
                if (ok) ord = o + p.size[j];
            }
            const unsigned same = __match_any_sync(0xffffffffu, ord);
            const int before = ok ? cnt[ord] : 0;
            __syncwarp();
            if (ok) {
                if (write) {
                    const int64_t sl = p.base[(int64_t)ord * p.n_units + u] + before + __popc(same & lt);
                    int32_t *dst = p.out + sl * (p.m + 1);
                    for (int q = 0; q < p.m; ++q) dst[q] = tp[q];
                    dst[p.m] = (int32_t)j;
                    p.out_order[sl] = ord;
                }
                if ((same & lt) == 0) cnt[ord] = before + __popc(same);   // group leader
            }
            __syncwarp();
        }
        if (!write)
            for (int q = lane; q <= p.K; q += 32) p.counts[(int64_t)q * p.n_units + u] = cnt[q];
        __syncwarp();
    }
}

__global__ void iota_order_kernel(int32_t *idx, int32_t *ord, const int32_t *size, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        idx[i] = (int32_t)i;
        ord[i] = size[i];
    }
}

int grid1(int64_t n, int block, int n_sm)
{
    int64_t g = (n + block - 1) / block;
    const int64_t cap = (int64_t)n_sm * 64;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

namespace {

template <typename T>
pne_status scan_to(pne_ctx *ctx, const T *src, int64_t *dst, int64_t n, int64_t *d_total, cudaStream_t s)
{
    if (n <= 0) { PNE_CUDA_TRY(ctx, cudaMemsetAsync(d_total, 0, 8, s)); return PNE_OK; }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb <= kOneBlockTiles) {
        {
            ProfScope ps__(ctx, s, "scan");
            scan_one_block_kernel<T><<<1, 1024, 0, s>>>(src, dst, n, d_total);
        }
        PNE_CUDA_TRY(ctx, cudaGetLastError());
        return PNE_OK;
    }
    DevBuf sums;
    pne_status st = dev_alloc(ctx, sums, (size_t)nb * 8, s);
    if (st) return st;
    int64_t *ts = (int64_t *)sums.ptr;
    {
        ProfScope ps__(ctx, s, "scan");
        scan_tiles_kernel<T><<<(unsigned)nb, 1024, 0, s>>>(src, dst, n, ts);
    }
    if (cudaGetLastError() != cudaSuccess) {
        dev_free(ctx, sums, s);
        set_error(ctx, PNE_ECUDA, "scan_tiles_kernel launch failed");
        return PNE_ECUDA;
    }
    if ((st = scan_to<int64_t>(ctx, ts, ts, nb, d_total, s))) { dev_free(ctx, sums, s); return st; }
    {
        ProfScope ps__(ctx, s, "scan");
        scan_add_tiles_kernel<<<(unsigned)nb, 1024, 0, s>>>(dst, n, ts);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    dev_free(ctx, sums, s);
    return PNE_OK;
}

}  // namespace

// exclusive scan (in place) of n int64 values; the total is written to d_total
// on the device (no synchronisation)
pne_status device_exclusive_scan_to(pne_ctx *ctx, int64_t *d, int64_t n, int64_t *d_total, cudaStream_t s)
{
    return scan_to<int64_t>(ctx, d, d, n, d_total, s);
}

// exclusive scan (in place) of n int64 values; the total is returned on the host
pne_status device_exclusive_scan(pne_ctx *ctx, int64_t *d, int64_t n, int64_t *h_total, cudaStream_t s)
{
    if (n == 0) { *h_total = 0; return PNE_OK; }
    DevBuf tot;
    pne_status st = dev_alloc(ctx, tot, 8, s);
    if (st) return st;
    if ((st = device_exclusive_scan_to(ctx, d, n, (int64_t *)tot.ptr, s))) { dev_free(ctx, tot, s); return st; }
    int64_t *h = pinned_i64(ctx, 1);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h, tot.ptr, 8, cudaMemcpyDeviceToHost, s));
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    *h_total = *h;
    dev_free(ctx, tot, s);
    return PNE_OK;
}

namespace {

// exclusive scan of n int32 counts into int64 dst; the total lands in d_total
pne_status scan_i32_to(pne_ctx *ctx, const int32_t *src, int64_t *dst, int64_t n, int64_t *d_total, cudaStream_t s)
{
    return scan_to<int32_t>(ctx, src, dst, n, d_total, s);
}

// counts [rows][cols] int32 -> base (exclusive scan, row-major) int64.  The
// row starts are gathered on the device and their copy to pinned memory is
// queued, together with `extra_bytes` from `extra_dev` (a multiple of 8);
// *h_out receives the pinned words (rows + 1 starts, then the extra bytes).
pne_status scan_counts_queue(pne_ctx *ctx, const int32_t *d_counts, int rows, int64_t cols, DevBuf &base,
                             cudaStream_t s, int64_t **h_out, const void *extra_dev = nullptr, size_t extra_bytes = 0)
{
    const int64_t n = (int64_t)rows * cols;
    pne_status st = dev_alloc(ctx, base, (size_t)(std::max<int64_t>(n, 1) + rows + 3) * 8, s);
    if (st) return st;
    int64_t *b = (int64_t *)base.ptr;
    int64_t *starts = b + std::max<int64_t>(n, 1);          // [rows + 1]
    int64_t *tot = starts + rows + 1;                       // [1]
    // exclusive scan; its total lands in tot
    if ((st = scan_i32_to(ctx, d_counts, b, n, tot, s))) return st;
    row_starts_kernel<<<(rows + 1 + 127) / 128, 128, 0, s>>>(b, rows, cols, n, starts, tot);
    PNE_LAUNCH_CHECK(ctx);
    const size_t words = (size_t)(rows + 1) + extra_bytes / 8;
    int64_t *h = pinned_i64(ctx, words);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h, starts, (rows + 1) * 8, cudaMemcpyDeviceToHost, s));
    if (extra_bytes)
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h + rows + 1, extra_dev, extra_bytes, cudaMemcpyDeviceToHost, s));
    *h_out = h;
    return PNE_OK;
}

// ... and the same with the wait: per-row totals into row_tot, the extra
// bytes into extra_host.
pne_status scan_counts(pne_ctx *ctx, const int32_t *d_counts, int rows, int64_t cols, DevBuf &base,
                       std::vector<int64_t> &row_tot, cudaStream_t s, const void *extra_dev = nullptr,
                       size_t extra_bytes = 0, void *extra_host = nullptr)
{
    int64_t *h = nullptr;
    pne_status st = scan_counts_queue(ctx, d_counts, rows, cols, base, s, &h, extra_dev, extra_bytes);
    if (st) return st;
    {
        HostScope hw__(ctx, "sync_counts");
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    row_tot.assign(rows, 0);
    for (int r = 0; r < rows; ++r) row_tot[r] = h[r + 1] - h[r];
    if (extra_bytes) std::memcpy(extra_host, h + rows + 1, extra_bytes);
    return PNE_OK;
}

void launch_expand(int pass, bool fuse, int G, cudaStream_t s, const GeomView &gv, const Arena &A, int lo, int hi,
                   int K, int mode, const Emit &o)
{
    const int T = 32 * kExpandWarps;
    switch (pass) {
    case kCount:
        if (fuse) expand_kernel<kCount, true><<<G, T, 0, s>>>(gv, A, lo, hi, K, mode, o);
        else expand_kernel<kCount, false><<<G, T, 0, s>>>(gv, A, lo, hi, K, mode, o);
        break;
    case kEmitCount: expand_kernel<kEmitCount, false><<<G, T, 0, s>>>(gv, A, lo, hi, K, mode, o); break;
    case kPairCount: expand_kernel<kPairCount, true><<<G, T, 0, s>>>(gv, A, lo, hi, K, mode, o); break;
    default:
        if (fuse) expand_kernel<kEmit, true><<<G, T, 0, s>>>(gv, A, lo, hi, K, mode, o);
        else expand_kernel<kEmit, false><<<G, T, 0, s>>>(gv, A, lo, hi, K, mode, o);
        break;
    }
}

}  // namespace

pne_status enumerate_clusters(pne_ctx *ctx, const Geometry &g, int K, int mode, EnumRecord &rec,
                              cudaStream_t s)
{
    const int Mc = g.n_bonds;
    rec.K = K; rec.mode = mode; rec.n_closed = Mc;
    rec.width = std::max(1, K);
    rec.vwidth = K + 1;
    int maxdeg = g.max_deg;
    const int umax_need = 2 * (maxdeg - 1) + K * (maxdeg - 1) + 2;
    if (K > 32 || umax_need > 128) {
        set_error(ctx, PNE_EINVAL, "expansion order too large for the cluster search");
        return PNE_EINVAL;
    }
    if ((kPrefixMax + 1) * (maxdeg - 1) > kNodeU) { set_error(ctx, PNE_EINVAL, "site degree too large"); return PNE_EINVAL; }
    GeomView gv{g.d_bond_site, g.d_site_ptr, g.d_site_bonds, g.d_site_nbr};
    // prefix levels 1..D are expanded breadth-first; the last one closes both
    // remaining sizes (LOOP mode, D == K - 2), only emits (D == K - 1) or is
    // searched depth-first (K - 1 > kPrefixMax)
    const bool fuse = mode == PNE_MODE_LOOP && K >= 3 && K - 2 <= kPrefixMax;
    const int D = fuse ? K - 2 : ((K <= 1) ? 1 : std::min(kPrefixMax, K - 1));
    const int final_kind = fuse ? 3 : ((K <= 1) ? 0 : (D == K - 1 ? 1 : 2));
    const bool small = (K <= 12 && umax_need <= 64);
    // chunks of the blocked passes: one wave of resident blocks (the occupancy
    // is queried once per context)
    if (ctx->occ_expand < 0) {
        int a = 0;
        PNE_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, expand_kernel<kCount, true>, 32 * kExpandWarps, 0));
        ctx->occ_expand = a;
    }
    const int G = ctx->n_sm * std::max(1, ctx->occ_expand.load());
    const int Gd = grid1(1 << 20, 128, ctx->n_sm);    // grid of the depth-first kernel
    const std::string hint_key = std::to_string(g.hash) + ":" + std::to_string(Mc) + ":" + std::to_string(K) + ":" +
                                 std::to_string(mode);
    int64_t cap = kArenaFirst;
    {
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        auto it = ctx->arena_hint.find(hint_key);
        if (it != ctx->arena_hint.end()) cap = it->second;
    }
    const int64_t cap_max = ctx->arena_max > 0 ? std::max<int64_t>(ctx->arena_max, Mc) : kNodeCap;
    cap = std::min(cap_max, std::max<int64_t>(cap, Mc));
    Emit none{nullptr, nullptr, nullptr, rec.width, rec.vwidth};
    auto dfs = [&](const Arena &A, int level, int write, const Emit &o) {
        ProfScope ps__(ctx, s, "enum_dfs");
        if (small) dfs_kernel<12, 64><<<Gd, 128, 0, s>>>(gv, A, level, K, mode, write, o);
        else dfs_kernel<32, 128><<<Gd, 128, 0, s>>>(gv, A, level, K, mode, write, o);
    };
    struct Readback { int64_t lv[kPrefixMax + 2]; SearchCtl ctl; } hb;
    DevBuf nodes, tables, counts, base;
    // the arena's buffers are released on every exit, behind the kernels
    // already queued on `s`
    struct Release {
        pne_ctx *ctx; cudaStream_t s; DevBuf *b[4];
        ~Release() { for (DevBuf *x : b) dev_free(ctx, *x, s); }
    } release_arena{ctx, s, {&nodes, &tables, &counts, &base}};
    Arena A{};
    std::vector<int64_t> per_size;
    int dfs_level = 0;
    pne_status st;
    for (;;) {
        // arena: nodes, then [lv, ctl | child_off | chunk_tot | gmask | emask | child_cnt], then counts
        if ((st = dev_alloc(ctx, nodes, sizeof(Node) * (size_t)cap, s))) return st;
        const size_t tab_bytes = sizeof(Readback) + (size_t)cap * 4 + (size_t)cap * 24 + (size_t)G * 8 + 64;
        if ((st = dev_alloc(ctx, tables, tab_bytes, s))) return st;
        if ((st = dev_alloc(ctx, counts, (size_t)(K + 1) * cap * 4, s))) return st;
        char *tb = (char *)tables.ptr;
        A.nodes = (Node *)nodes.ptr;
        A.cap = cap;
        A.lv = (int64_t *)tb;
        A.ctl = (SearchCtl *)(tb + offsetof(Readback, ctl));
        A.child_off = (int64_t *)(tb + sizeof(Readback));
        A.chunk_tot = A.child_off + cap;
        A.gmask = reinterpret_cast<uint64_t *>(A.chunk_tot + G);
        A.emask = A.gmask + cap;
        A.child_cnt = (int32_t *)(A.emask + cap);
        A.counts = (int32_t *)counts.ptr;
        A.base = nullptr;
        PNE_CUDA_TRY(ctx, cudaMemsetAsync(counts.ptr, 0, (size_t)(K + 1) * cap * 4, s));
        arena_init_kernel<<<1, 32, 0, s>>>(A, Mc);
        PNE_LAUNCH_CHECK(ctx);
        {
            ProfScope ps__(ctx, s, "enum_roots");
            roots_kernel<<<grid1(Mc, 128, ctx->n_sm), 128, 0, s>>>(gv, Mc, mode, A, none, 0);
        }
        PNE_LAUNCH_CHECK(ctx);
        // each pass is its own kernel and is timed under its own name
        for (int d = 1; d < D; ++d) {
            {
                ProfScope ps__(ctx, s, "enum_count");
                launch_expand(kCount, final_kind == 3, G, s, gv, A, d, d, K, mode, none);
            }
            PNE_LAUNCH_CHECK(ctx);
            {
                ProfScope ps__(ctx, s, "enum_children");
                expand_children_kernel<<<G, 32 * kExpandWarps, 0, s>>>(gv, A, d, K, mode);
            }
            PNE_LAUNCH_CHECK(ctx);
        }
        if (final_kind == 1 || final_kind == 3) {
            ProfScope ps__(ctx, s, "enum_close_count");
            launch_expand(final_kind == 3 ? kPairCount : kEmitCount, final_kind == 3, G, s, gv, A, D, D, K, mode, none);
        } else if (final_kind == 2) {
            dfs(A, D, 0, none);
        }
        PNE_LAUNCH_CHECK(ctx);
        // one (size, node) table over the arena; the same round trip brings the
        // level bounds and the stop record
        if ((st = scan_counts(ctx, A.counts, K + 1, cap, base, per_size, s, A.lv, sizeof(Readback), &hb))) return st;
        if (hb.ctl.cand_overflow) {
            set_error(ctx, PNE_EOVERFLOW, "candidate list overflow in the cluster search");
            return PNE_EOVERFLOW;
        }
        if (hb.ctl.stop == 0) { dfs_level = (final_kind == 2) ? D : 0; break; }
        if (cap < cap_max) {
            // the tree outgrew the arena: grow it and search again
            cap = std::min(cap_max, std::max(4 * cap, 2 * hb.ctl.need));
            dev_free(ctx, nodes, s); dev_free(ctx, tables, s); dev_free(ctx, counts, s); dev_free(ctx, base, s);
            continue;
        }
        // the largest arena holds levels 1..stop: search below level `stop` depth-first
        dfs_level = hb.ctl.stop;
        dfs(A, dfs_level, 0, none);
        PNE_LAUNCH_CHECK(ctx);
        dev_free(ctx, base, s);
        if ((st = scan_counts(ctx, A.counts, K + 1, cap, base, per_size, s))) return st;
        break;
    }
    {
        // the next search of this geometry starts with an arena that fits
        const int last = hb.ctl.stop ? hb.ctl.stop : D;
        const int64_t used = ((hb.lv[last] + 1023) / 1024) * 1024;
        std::lock_guard<std::mutex> lk(ctx->cache_mu);
        ctx->arena_hint[hint_key] = std::min(cap_max, std::max<int64_t>(used, 1024));
    }
    uint64_t n_cl = 0;
    rec.size_start.assign(K + 2, 0);
    for (int q = 0; q <= K; ++q) { rec.size_start[q] = (int64_t)n_cl; n_cl += per_size[q]; }
    rec.size_start[K + 1] = (int64_t)n_cl;
    rec.n_clusters = n_cl;
    const size_t nn = std::max<uint64_t>(n_cl, 1);
    if ((st = dev_alloc(ctx, rec.cl_edges, nn * rec.width * 4, s))) return st;
    if ((st = dev_alloc(ctx, rec.cl_verts, nn * rec.vwidth * 4, s))) return st;
    if ((st = dev_alloc(ctx, rec.cl_size, nn * 4, s))) return st;
    Emit out{(int32_t *)rec.cl_edges.ptr, (int32_t *)rec.cl_verts.ptr, (int32_t *)rec.cl_size.ptr, rec.width, rec.vwidth};
    A.base = (const int64_t *)base.ptr;
    // write passes: the anchors (ALL mode), the breadth-first emissions of
    // levels 1..last_bfs, and the depth-first subtrees
    const int last_bfs = dfs_level ? dfs_level - 1 : ((final_kind == 1 || final_kind == 3) ? D : 0);
    if (mode == PNE_MODE_ALL) {
        ProfScope ps__(ctx, s, "enum_roots");
        roots_kernel<<<grid1(Mc, 128, ctx->n_sm), 128, 0, s>>>(gv, Mc, mode, A, out, 1);
    }
    PNE_LAUNCH_CHECK(ctx);
    if (last_bfs >= 1) {
        ProfScope ps__(ctx, s, "enum_emit");
        launch_expand(kEmit, final_kind == 3 && dfs_level == 0, G, s, gv, A, 1, last_bfs, K, mode, out);
    }
    PNE_LAUNCH_CHECK(ctx);
    if (dfs_level) dfs(A, dfs_level, 1, out);
    PNE_LAUNCH_CHECK(ctx);
    return PNE_OK;
}

namespace {

// Counting half of one tuple round (input tuples of length tp.m): the unit
// offsets, the counting pass and the queued readback of the (order, unit)
// row starts.
pne_status tuple_round_count(pne_ctx *ctx, EnumRecord &rec, TuplePrep &tp, cudaStream_t s)
{
    const int K = rec.K, m = tp.m;
    TupleParams p;
    p.verts = (const int32_t *)rec.cl_verts.ptr; p.size = (const int32_t *)rec.cl_size.ptr;
    p.vwidth = rec.vwidth; p.K = K; p.m = m;
    p.in = (const int32_t *)tp.in_idx.ptr; p.in_order = (const int32_t *)tp.in_ord.ptr; p.n_in = tp.n_in;
    p.size_end = (const int64_t *)tp.d_size_end.ptr;
    p.counts = nullptr; p.base = nullptr; p.out = nullptr; p.out_order = nullptr;
    pne_status st;
    if ((st = dev_alloc(ctx, tp.uoff, (tp.n_in + 1) * 8, s))) return st;
    int64_t n_units = 0;
    if (m == 1) {
        // pairs: input tuple i is cluster i, whose size (hence the candidate
        // range) the host knows from the size-grouped list
        std::vector<int64_t> h_off(tp.n_in + 1, 0);
        for (int q = 1; q <= K; ++q)
            for (int64_t i = rec.size_start[q]; i < std::min<int64_t>(rec.size_start[q + 1], tp.n_in); ++i) {
                const int64_t lo = i + 1, hi = (q < K) ? tp.size_end[K - q] : lo;
                h_off[i] = hi > lo ? (hi - lo + kTupleChunk - 1) / kTupleChunk : 0;
            }
        for (int64_t i = 0; i < tp.n_in; ++i) { const int64_t c = h_off[i]; h_off[i] = n_units; n_units += c; }
        h_off[tp.n_in] = n_units;
        if ((st = upload(ctx, tp.uoff.ptr, h_off.data(), (tp.n_in + 1) * 8, s))) return st;
    } else {
        {
            ProfScope ps__(ctx, s, "enum_terms");
            tuple_chunks_kernel<<<grid1(tp.n_in, 256, ctx->n_sm), 256, 0, s>>>(p, (int64_t *)tp.uoff.ptr);
        }
        PNE_LAUNCH_CHECK(ctx);
        if ((st = device_exclusive_scan(ctx, (int64_t *)tp.uoff.ptr, tp.n_in, &n_units, s))) return st;
    }
    tp.n_units = n_units;
    p.unit_off = (const int64_t *)tp.uoff.ptr; p.n_units = n_units;
    tp.tsmem = (size_t)kTupleWarps * (m * rec.vwidth + kMaxOrder + 1) * 4;
    tp.h = nullptr;
    if (n_units > 0) {
        if ((st = dev_alloc(ctx, tp.counts, (size_t)(K + 1) * n_units * 4, s))) return st;
        p.counts = (int32_t *)tp.counts.ptr;
        {
            ProfScope ps__(ctx, s, "enum_terms");
            tuple_kernel<<<grid1(n_units, kTupleWarps, ctx->n_sm), 32 * kTupleWarps, tp.tsmem, s>>>(p, 0);
        }
        PNE_CUDA_TRY(ctx, cudaGetLastError());
        if ((st = scan_counts_queue(ctx, (const int32_t *)tp.counts.ptr, K + 1, n_units, tp.base, s, &tp.h))) return st;
    }
    return PNE_OK;
}

// Writing half: waits for the row starts, writes the round's tuples (a new
// level of terms) and makes them the next round's input.
pne_status tuple_round_write(pne_ctx *ctx, EnumRecord &rec, TuplePrep &tp, cudaStream_t s)
{
    const int K = rec.K, m = tp.m;
    std::vector<int64_t> per_order(K + 1, 0);
    if (tp.h) {
        {
            HostScope hw__(ctx, "sync_counts");
            PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        }
        for (int r = 0; r <= K; ++r) per_order[r] = tp.h[r + 1] - tp.h[r];
        tp.h = nullptr;
    }
    EnumRecord::Level L;
    L.m = m + 1;
    L.order_start.assign(K + 2, 0);
    int64_t n_out = 0;
    for (int q = 0; q <= K; ++q) { L.order_start[q] = n_out; n_out += per_order[q]; }
    L.order_start[K + 1] = n_out;
    L.n = (uint64_t)n_out;
    DevBuf out_ord;
    pne_status st;
    if (n_out > 0) {
        if ((st = dev_alloc(ctx, L.idx, (size_t)n_out * (m + 1) * 4, s))) return st;
        if ((st = dev_alloc(ctx, out_ord, (size_t)n_out * 4, s))) return st;
        TupleParams p;
        p.verts = (const int32_t *)rec.cl_verts.ptr; p.size = (const int32_t *)rec.cl_size.ptr;
        p.vwidth = rec.vwidth; p.K = K; p.m = m;
        p.in = (const int32_t *)tp.in_idx.ptr; p.in_order = (const int32_t *)tp.in_ord.ptr; p.n_in = tp.n_in;
        p.size_end = (const int64_t *)tp.d_size_end.ptr;
        p.unit_off = (const int64_t *)tp.uoff.ptr; p.n_units = tp.n_units;
        p.counts = (int32_t *)tp.counts.ptr;
        p.base = (const int64_t *)tp.base.ptr;
        p.out = (int32_t *)L.idx.ptr; p.out_order = (int32_t *)out_ord.ptr;
        {
            ProfScope ps__(ctx, s, "enum_terms");
            tuple_kernel<<<grid1(tp.n_units, kTupleWarps, ctx->n_sm), 32 * kTupleWarps, tp.tsmem, s>>>(p, 1);
        }
        PNE_CUDA_TRY(ctx, cudaGetLastError());
    }
    for (int q = 0; q <= K; ++q) rec.terms_by_order[q] += per_order[q];
    rec.n_terms += (uint64_t)n_out;
    dev_free(ctx, tp.uoff, s); dev_free(ctx, tp.counts, s); dev_free(ctx, tp.base, s);
    if (tp.in_owned) dev_free(ctx, tp.in_idx, s);
    dev_free(ctx, tp.in_ord, s);
    if (n_out > 0) rec.levels.push_back(L);
    tp.in_idx = L.idx; tp.in_owned = false;     // the level keeps ownership
    tp.in_ord = out_ord;
    tp.n_in = n_out;
    tp.m = m + 1;
    return PNE_OK;
}

}  // namespace

pne_status tuples_begin(pne_ctx *ctx, EnumRecord &rec, TuplePrep &tp, cudaStream_t s)
{
    const int K = rec.K;
    tp = TuplePrep();
    rec.levels.clear();
    rec.terms_by_order.assign(K + 1, 0);
    rec.terms_by_order[0] = 1;
    for (int q = 1; q <= K; ++q) rec.terms_by_order[q] += rec.size_start[q + 1] - rec.size_start[q];
    for (int q = 1; q <= K; ++q) if (rec.size_start[q + 1] > rec.size_start[q]) { tp.s_min = q; break; }
    rec.n_terms = 1 + rec.n_clusters;
    if (tp.s_min == 0 || rec.n_clusters == 0) return PNE_OK;
    // size_end[q] = first cluster index with size > q
    tp.size_end.assign(K + 2, 0);
    for (int q = 0; q <= K; ++q) tp.size_end[q] = rec.size_start[q + 1];
    tp.size_end[K + 1] = rec.size_start[K + 1];
    pne_status st;
    if ((st = dev_alloc(ctx, tp.d_size_end, (K + 2) * 8, s))) return st;
    if ((st = upload(ctx, tp.d_size_end.ptr, tp.size_end.data(), (K + 2) * 8, s))) return st;
    // first round: every cluster that can start a pair (size <= K - s_min)
    tp.n_in = (K - tp.s_min >= tp.s_min) ? tp.size_end[K - tp.s_min] : 0;
    tp.m = 1;
    if (tp.n_in > 0) {
        if ((st = dev_alloc(ctx, tp.in_idx, tp.n_in * 4, s))) return st;
        if ((st = dev_alloc(ctx, tp.in_ord, tp.n_in * 4, s))) return st;
        {
            ProfScope ps__(ctx, s, "enum_terms");
            iota_order_kernel<<<grid1(tp.n_in, 256, ctx->n_sm), 256, 0, s>>>((int32_t *)tp.in_idx.ptr,
                                                                          (int32_t *)tp.in_ord.ptr,
                                                                          (const int32_t *)rec.cl_size.ptr, tp.n_in);
        }
        PNE_LAUNCH_CHECK(ctx);
        if (2 * tp.s_min <= K) {
            if ((st = tuple_round_count(ctx, rec, tp, s))) return st;
            tp.active = true;
        }
    }
    return PNE_OK;
}

pne_status tuples_finish(pne_ctx *ctx, EnumRecord &rec, TuplePrep &tp, cudaStream_t s)
{
    const int K = rec.K;
    pne_status st;
    while (tp.active) {
        if ((st = tuple_round_write(ctx, rec, tp, s))) return st;
        tp.active = tp.n_in > 0 && (tp.m + 1) * tp.s_min <= K;
        if (tp.active && (st = tuple_round_count(ctx, rec, tp, s))) return st;
    }
    if (tp.in_owned) dev_free(ctx, tp.in_idx, s);
    dev_free(ctx, tp.in_ord, s);
    dev_free(ctx, tp.d_size_end, s);
    return PNE_OK;
}

void tuples_abort(pne_ctx *ctx, TuplePrep &tp, cudaStream_t s)
{
    DevBuf *bufs[] = {&tp.d_size_end, &tp.in_ord, &tp.uoff, &tp.counts, &tp.base};
    for (DevBuf *b : bufs) dev_free(ctx, *b, s);
    if (tp.in_owned) dev_free(ctx, tp.in_idx, s);
    tp.active = false;
}

pne_status enumerate_tuples(pne_ctx *ctx, EnumRecord &rec, cudaStream_t s)
{
    TuplePrep tp;
    pne_status st = tuples_begin(ctx, rec, tp, s);
    return st ? st : tuples_finish(ctx, rec, tp, s);
}

}  // namespace pne
