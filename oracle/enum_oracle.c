/* Oracle cluster enumeration in plain C (FP-free, integer only).
 *
 * TEST INFRASTRUCTURE ONLY: called from oracle/enumerate.py; never linked into
 * or called by the product library.
 *
 * A cluster is a connected set C of closed bonds (Sec. III.A: a connected
 * configuration of excited indices).  In LOOP mode C may contain no vertex of
 * C-degree exactly one: such a "dangling excitation" makes the term vanish at a
 * BP fixed point (Sec. III.A and III.B).  In ALL mode every connected set is
 * kept.  Open bonds (second site < 0) are never partitioned and are skipped.
 *
 * Two independent methods, both plain:
 *   oracle_enum_bitmask  every subset of the closed bonds (at most 30 of them)
 *                        is tested directly for size, connectivity and degree;
 *   oracle_enum_grow     for every anchor bond a, level-by-level growth of the
 *                        connected sets whose smallest bond is a: each set of
 *                        size s is extended by every adjacent bond > a, and the
 *                        extensions are sorted and de-duplicated.  Sets that
 *                        have more degree-1 vertices than 2*(K - s) are dropped,
 *                        since each further bond can repair at most two.
 * Output rows: the sorted bond ids of one cluster, padded with -1 to `width`.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* bitmask scan                                                        */
/* ------------------------------------------------------------------ */
int64_t oracle_enum_bitmask(int32_t n_sites, int32_t n_bonds, const int32_t *bond_site,
                            int32_t K, int32_t mode, int32_t width,
                            int32_t *out, int64_t cap)
{
    int32_t closed[64];
    int nc = 0;
    for (int b = 0; b < n_bonds; ++b)
        if (bond_site[2 * b + 1] >= 0) {
            if (nc == 30) return -1;
            closed[nc++] = b;
        }
    if (n_sites > 64) return -1;
    uint64_t vm[30];
    for (int i = 0; i < nc; ++i) {
        int b = closed[i];
        vm[i] = (1ull << bond_site[2 * b]) | (1ull << bond_site[2 * b + 1]);
    }
    int deg[64];
    memset(deg, 0, sizeof deg);
    int64_t count = 0;
    uint64_t nmask = 1ull << nc;
    for (uint64_t m = 1; m < nmask; ++m) {
        int k = __builtin_popcountll(m);
        if (k > K) continue;
        /* degree test (LOOP mode): a vertex of degree one rejects the set */
        if (mode == 0) {
            int bad = 0;
            for (uint64_t r = m; r; r &= r - 1) {
                int b = closed[__builtin_ctzll(r)];
                deg[bond_site[2*b]]++; deg[bond_site[2*b+1]]++;
            }
            for (uint64_t r = m; r; r &= r - 1) {
                int b = closed[__builtin_ctzll(r)];
                if (deg[bond_site[2*b]] == 1 || deg[bond_site[2*b+1]] == 1) bad = 1;
            }
            for (uint64_t r = m; r; r &= r - 1) {
                int b = closed[__builtin_ctzll(r)];
                deg[bond_site[2*b]] = 0; deg[bond_site[2*b+1]] = 0;
            }
            if (bad) continue;
        }
        /* connectivity: grow the vertex set from the lowest bond until stable */
        int first = __builtin_ctzll(m);
        uint64_t cover = vm[first], all = 0;
        for (uint64_t r = m; r; r &= r - 1) all |= vm[__builtin_ctzll(r)];
        for (;;) {
            uint64_t prev = cover;
            for (uint64_t r = m; r; r &= r - 1) {
                int i = __builtin_ctzll(r);
                if (vm[i] & cover) cover |= vm[i];
            }
            if (cover == prev) break;
        }
        if (cover != all) continue;
        if (count < cap) {
            int32_t *row = out + count * (int64_t)width;
            int j = 0;
            for (int i = 0; i < nc; ++i) if (m >> i & 1) row[j++] = closed[i];
            for (; j < width; ++j) row[j] = -1;
        }
        ++count;
    }
    return count;
}

/* number of subsets of the closed bonds, by size, in which every vertex has
 * even degree (the Ising high-temperature graphs), by Gray-code traversal */
int32_t oracle_even_subsets_by_size(int32_t n_sites, int32_t n_bonds, const int32_t *bond_site,
                                    int64_t *counts /* [n_closed + 1] */)
{
    int32_t closed[64];
    int nc = 0;
    for (int b = 0; b < n_bonds; ++b)
        if (bond_site[2 * b + 1] >= 0) { if (nc == 34) return -1; closed[nc++] = b; }
    if (n_sites > 64) return -1;
    uint64_t vm[34];
    for (int i = 0; i < nc; ++i) {
        int b = closed[i];
        vm[i] = (1ull << bond_site[2 * b]) | (1ull << bond_site[2 * b + 1]);
    }
    for (int i = 0; i <= nc; ++i) counts[i] = 0;
    uint64_t parity = 0, mask = 0;
    int size = 0;
    counts[0] = 1;
    uint64_t n = 1ull << nc;
    for (uint64_t g = 1; g < n; ++g) {
        int i = __builtin_ctzll(g);            /* bit flipped by the Gray code */
        mask ^= 1ull << i;
        parity ^= vm[i];
        size += (mask >> i & 1) ? 1 : -1;
        if (parity == 0) counts[size]++;
    }
    return nc;
}

/* ------------------------------------------------------------------ */
/* per-anchor level growth                                             */
/* ------------------------------------------------------------------ */
typedef struct { int32_t *v; int64_t n, cap; } ivec;

static int ivec_push(ivec *a, const int32_t *x, int w)
{
    if (a->n + w > a->cap) {
        int64_t nc = a->cap ? a->cap * 2 : 1024;
        while (nc < a->n + w) nc *= 2;
        int32_t *p = (int32_t *)realloc(a->v, (size_t)nc * sizeof(int32_t));
        if (!p) return -1;
        a->v = p; a->cap = nc;
    }
    memcpy(a->v + a->n, x, (size_t)w * sizeof(int32_t));
    a->n += w;
    return 0;
}

static int g_width;
static int cmp_rows(const void *a, const void *b)
{
    return memcmp(a, b, (size_t)g_width * sizeof(int32_t));
}
/* memcmp on int32 orders by bytes, which is not numeric order, but any total
 * order serves for de-duplication; callers re-sort by value. */

/* number of vertices of degree one in a bond set */
static int dangling(const int32_t *S, int s, const int32_t *bond_site, int32_t *vtx, int32_t *dg)
{
    int nv = 0;
    for (int i = 0; i < s; ++i)
        for (int e = 0; e < 2; ++e) {
            int x = bond_site[2 * S[i] + e], j;
            for (j = 0; j < nv; ++j) if (vtx[j] == x) break;
            if (j == nv) { vtx[nv] = x; dg[nv] = 0; ++nv; }
            dg[j]++;
        }
    int d = 0;
    for (int j = 0; j < nv; ++j) d += (dg[j] == 1);
    return d;
}

/* Growth from anchor bond a (every connected set whose smallest bond is a),
 * level by level with sort/unique de-duplication; each set kept by the mode
 * is passed to emit().  Returns 0, or -2 when memory ran out. */
typedef void (*emit_fn)(const int32_t *S, int s, void *user);

static int grow_anchor(int a, const int32_t *bond_site, const int32_t *site_ptr, const int32_t *site_bonds,
                       int32_t K, int32_t mode, ivec *cur, ivec *nxt, emit_fn emit, void *user)
{
    int32_t vtx[2 * 64], dg[2 * 64], tmp[64];
    cur->n = 0;
    int32_t one = a;
    if (ivec_push(cur, &one, 1)) return -2;
    for (int s = 1; s <= K; ++s) {
        int64_t nsets = cur->n / s;
        /* emit this level */
        for (int64_t r = 0; r < nsets; ++r) {
            const int32_t *S = cur->v + r * s;
            int d = dangling(S, s, bond_site, vtx, dg);
            if (mode == 0 && d != 0) continue;
            emit(S, s, user);
        }
        if (s == K) break;
        /* grow to level s + 1 */
        nxt->n = 0;
        for (int64_t r = 0; r < nsets; ++r) {
            const int32_t *S = cur->v + r * s;
            for (int i = 0; i < s; ++i)
                for (int e = 0; e < 2; ++e) {
                    int x = bond_site[2 * S[i] + e];
                    for (int p = site_ptr[x]; p < site_ptr[x + 1]; ++p) {
                        int f = site_bonds[p];
                        if (f <= a || bond_site[2 * f + 1] < 0) continue;
                        int in = 0;
                        for (int j = 0; j < s; ++j) if (S[j] == f) { in = 1; break; }
                        if (in) continue;
                        /* sorted insert of f */
                        int j = 0, t = 0;
                        while (j < s && S[j] < f) tmp[t++] = S[j++];
                        tmp[t++] = f;
                        while (j < s) tmp[t++] = S[j++];
                        if (mode == 0) {
                            int d = dangling(tmp, s + 1, bond_site, vtx, dg);
                            if (d > 2 * (K - (s + 1))) continue;
                        }
                        if (ivec_push(nxt, tmp, s + 1)) return -2;
                    }
                }
        }
        int64_t nn = nxt->n / (s + 1);
        g_width = s + 1;
        qsort(nxt->v, (size_t)nn, (size_t)(s + 1) * sizeof(int32_t), cmp_rows);
        int64_t u = 0;
        for (int64_t r = 0; r < nn; ++r) {
            if (u > 0 && memcmp(nxt->v + (u - 1) * (s + 1), nxt->v + r * (s + 1),
                                (size_t)(s + 1) * sizeof(int32_t)) == 0) continue;
            if (u != r) memmove(nxt->v + u * (s + 1), nxt->v + r * (s + 1), (size_t)(s + 1) * sizeof(int32_t));
            ++u;
        }
        nxt->n = u * (s + 1);
        ivec t2 = *cur; *cur = *nxt; *nxt = t2;
        if (cur->n == 0) break;
    }
    return 0;
}

struct rows_out { int32_t *out; int64_t cap, count; int width; };

static void emit_row(const int32_t *S, int s, void *user)
{
    struct rows_out *o = (struct rows_out *)user;
    if (o->count < o->cap) {
        int32_t *row = o->out + o->count * (int64_t)o->width;
        memcpy(row, S, (size_t)s * sizeof(int32_t));
        for (int j = s; j < o->width; ++j) row[j] = -1;
    }
    ++o->count;
}

int64_t oracle_enum_grow(int32_t n_sites, int32_t n_bonds, const int32_t *bond_site,
                         const int32_t *site_ptr, const int32_t *site_bonds,
                         int32_t K, int32_t mode, int32_t width,
                         int32_t *out, int64_t cap)
{
    (void)n_sites;
    if (K < 1 || width < K || K > 60) return -1;
    ivec cur = {0}, nxt = {0};
    struct rows_out o = {out, cap, 0, width};
    for (int a = 0; a < n_bonds; ++a) {
        if (bond_site[2 * a + 1] < 0) continue;
        if (grow_anchor(a, bond_site, site_ptr, site_bonds, K, mode, &cur, &nxt, emit_row, &o)) {
            free(cur.v); free(nxt.v); return -2;
        }
    }
    free(cur.v); free(nxt.v);
    return o.count;
}

struct counts_out { const int32_t *bond_site; int64_t *by_size, *even_by_size; };

static void emit_count(const int32_t *S, int s, void *user)
{
    struct counts_out *o = (struct counts_out *)user;
    o->by_size[s]++;
    if (!o->even_by_size) return;
    /* every vertex of even degree in the set (an even subgraph) */
    int32_t vtx[2 * 64], dg[2 * 64];
    int nv = 0;
    for (int i = 0; i < s; ++i)
        for (int e = 0; e < 2; ++e) {
            int x = o->bond_site[2 * S[i] + e], j;
            for (j = 0; j < nv; ++j) if (vtx[j] == x) break;
            if (j == nv) { vtx[nv] = x; dg[nv] = 0; ++nv; }
            dg[j]++;
        }
    for (int j = 0; j < nv; ++j) if (dg[j] & 1) return;
    o->even_by_size[s]++;
}

/* The same growth for the anchors a0 <= a < a1 only, counting the kept sets
 * by size into by_size[0..K] (no list is written), and, when even_by_size is
 * given, those whose every vertex has even degree into even_by_size[0..K]:
 * independent anchor ranges can be counted side by side and added up. */
int32_t oracle_count_grow_range(int32_t n_sites, int32_t n_bonds, const int32_t *bond_site,
                                const int32_t *site_ptr, const int32_t *site_bonds,
                                int32_t K, int32_t mode, int32_t a0, int32_t a1, int64_t *by_size,
                                int64_t *even_by_size)
{
    (void)n_sites;
    if (K < 1 || K > 60 || a0 < 0 || a1 > n_bonds) return -1;
    ivec cur = {0}, nxt = {0};
    struct counts_out o = {bond_site, by_size, even_by_size};
    for (int a = a0; a < a1; ++a) {
        if (bond_site[2 * a + 1] < 0) continue;
        if (grow_anchor(a, bond_site, site_ptr, site_bonds, K, mode, &cur, &nxt, emit_count, &o)) {
            free(cur.v); free(nxt.v); return -2;
        }
    }
    free(cur.v); free(nxt.v);
    return 0;
}
