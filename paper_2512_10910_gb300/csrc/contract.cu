// Cluster contractions and the per-order term sums.
//
// In the symmetrised gauge (App. B) every partitioned bond has P = e0 e0^T and
// Q = diag(0, 1, .., 1).  A cluster C (a connected set of excited bonds)
// therefore contracts to
//     Z'_C = sum over excited values alpha_e in 1..d_e-1 on C's bonds of
//            prod_{v in C} T'_v[alpha on v's C-legs, 0 on its other legs],
// i.e. one dense excitation block per site (the blocked layout).  Each site
// tensor is pre-divided by z_v (its all-zero entry), so the contraction gives
// w(C) = Z'_C / prod z_v directly (Sec. III.A: the term of a P/Q string is the
// vacuum times one factor per excited cluster).
//
// General clusters: one warp per cluster.  Sites are absorbed one at a time in
// a greedy order that keeps the open frontier (bonds with exactly one absorbed
// end) small; the intermediate tensor over the frontier lives in shared memory
// and is renormalised by a power of two after every step, the exponent being
// carried separately (a per-cluster log scale).  Precision: FP64, or FP32 /
// TF32-rounded / BF16 inputs with FP32 accumulation.
// Bond dimension 2 everywhere (one excited value per bond): each site
// contributes one number and a cluster is a plain product, one thread each.
//
// Term sums (Eq. A4, truncated at order K): a term is a tuple of vertex-
// disjoint clusters; its value divided by the vacuum is the product of their
// w.  Terms are stored grouped by order, and each order's sum is formed in
// FP64 by a fixed reduction tree (chunks of a fixed size, then chunk partials
// in index order), so results do not depend on scheduling.
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "pne_internal.h"

namespace pne {

namespace {

constexpr int kCtWarps = 4;          // warps per block, general contraction
constexpr int kMaxSteps = 32;        // sites per cluster in the general kernel
constexpr int kMaxFront = 12;        // frontier bonds
constexpr int kMaxClose = kMaxDeg;
constexpr int kStepInts = 8 + 4 * kMaxFront + 4 * kMaxClose;   // + float reciprocals of the dims

struct ContractParams {
    int64_t n_clusters;
    int n_members, n_sites;
    int width, vwidth;
    const int32_t *cl_edges, *cl_verts, *cl_size;
    const int32_t *bond_site, *bond_dim, *bond_leg;   // closed geometry
    const int32_t *blk_off;                           // [n_sites][64]
    const int64_t *tens_off;
    int64_t stride;                                   // entries per member
    const void *M;                                    // double / float / bf16
    const double *scale;                              // [members][n_sites]
    const int8_t *zero;                               // [members][n_sites]
    double *w;                                        // [members][n_clusters]
    int32_t *nzc;                                     // [members][n_clusters]
    int32_t *status;                                  // [0] buffer overflow
};

template <typename T> struct Load;
template <> struct Load<double> {
    static __device__ __forceinline__ double get(const void *p, int64_t i) { return ((const double *)p)[i]; }
};
template <> struct Load<float> {
    static __device__ __forceinline__ float get(const void *p, int64_t i) { return ((const float *)p)[i]; }
};
struct LoadBF16 {
    static __device__ __forceinline__ float get(const void *p, int64_t i)
    {
        return __bfloat162float(((const __nv_bfloat16 *)p)[i]);
    }
};

__device__ __forceinline__ float rnd_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// operand rounding of the intermediate tensor: 0 none, 1 TF32, 2 BF16
template <int R> __device__ __forceinline__ float rnd(float x)
{
    if (R == 1) return rnd_tf32(x);
    if (R == 2) return __bfloat162float(__float2bfloat16_rn(x));
    return x;
}
template <int R> __device__ __forceinline__ double rnd(double x) { return x; }

__device__ __forceinline__ double pow2(int e) { return ldexp(1.0, e); }

// ---------------------------------------------------------------- plan
// Step layout (ints): [0] site, [1] mask, [2] nF (size of the new frontier),
// [3] nC (closing bonds), [4] out_size, [5] close_size, [6] slot, [7] spare,
// then dimsF[kMaxFront], sxF[kMaxFront], smF[kMaxFront],
// dimsC[kMaxClose], sxC[kMaxClose], smC[kMaxClose], then the float bits of
// 1/dimsF[kMaxFront] and 1/dimsC[kMaxClose] for divide-free decoding.
// Builds the elimination plan of one cluster (single thread).  Returns the
// number of steps, or -1 when a limit is exceeded.
__device__ int build_plan(const ContractParams &P, int64_t c, int *plan, int *sites_out,
                          int maxT)
{
    const int32_t *E = P.cl_edges + c * P.width;
    const int32_t *V = P.cl_verts + c * P.vwidth;
    int s = 0;
    while (s < P.width && E[s] >= 0) ++s;
    int nv = 0;
    while (nv < P.vwidth && V[nv] >= 0) ++nv;
    if (nv > kMaxSteps) return -1;
    // per vertex: leg -> local edge index
    int legedge[kMaxSteps][kMaxDeg];
    int mask[kMaxSteps];
    for (int i = 0; i < nv; ++i) { mask[i] = 0; for (int l = 0; l < kMaxDeg; ++l) legedge[i][l] = -1; }
    int ends[32][2];
    int qd[32];
    for (int k = 0; k < s; ++k) {
        const int e = E[k];
        qd[k] = P.bond_dim[e] - 1;
        for (int side = 0; side < 2; ++side) {
            const int x = P.bond_site[2 * e + side];
            int lo = 0, hi = nv - 1, slot = -1;
            while (lo <= hi) { int mid = (lo + hi) >> 1; if (V[mid] == x) { slot = mid; break; } if (V[mid] < x) lo = mid + 1; else hi = mid - 1; }
            if (slot < 0) return -1;
            ends[k][side] = slot;
            const int leg = P.bond_leg[2 * e + side];
            legedge[slot][leg] = k;
            mask[slot] |= 1 << leg;
        }
    }
    bool visited[kMaxSteps];
    for (int i = 0; i < nv; ++i) visited[i] = false;
    int F[kMaxFront], nF = 0;
    for (int t = 0; t < nv; ++t) {
        // greedy choice: smallest new frontier, then smallest work, then lowest slot
        int best = -1, bestF = 1 << 30, bestW = 1 << 30;
        for (int i = 0; i < nv; ++i) {
            if (visited[i]) continue;
            int closing = 0, nnew = 0;
            for (int l = 0; l < kMaxDeg; ++l) {
                const int k = legedge[i][l];
                if (k < 0) continue;
                const int other = ends[k][0] == i ? ends[k][1] : ends[k][0];
                if (visited[other]) ++closing; else ++nnew;
            }
            const int f = nF - closing + nnew, wk = nF + nnew;
            if (f < bestF || (f == bestF && wk < bestW)) { best = i; bestF = f; bestW = wk; }
        }
        const int v = best;
        visited[v] = true;
        int *st = plan + t * kStepInts;
        int *dimsF = st + 8, *sxF = dimsF + kMaxFront, *smF = sxF + kMaxFront;
        int *dimsC = smF + kMaxFront, *sxC = dimsC + kMaxClose, *smC = sxC + kMaxClose;
        // strides of v's block: row-major over its C-legs, ascending leg order
        int mstride[kMaxDeg];
        {
            int mul = 1;
            for (int l = kMaxDeg - 1; l >= 0; --l)
                if (legedge[v][l] >= 0) { mstride[l] = mul; mul *= qd[legedge[v][l]]; }
        }
        // strides of the current X: row-major over F
        int xstride[kMaxFront];
        {
            int mul = 1;
            for (int i = nF - 1; i >= 0; --i) { xstride[i] = mul; mul *= qd[F[i]]; }
        }
        int F2[kMaxFront], n2 = 0, nC = 0;
        for (int i = 0; i < nF; ++i) {
            const int k = F[i];
            int leg = -1;
            for (int l = 0; l < kMaxDeg; ++l) if (legedge[v][l] == k) leg = l;
            if (leg >= 0) {                       // closing
                dimsC[nC] = qd[k]; sxC[nC] = xstride[i]; smC[nC] = mstride[leg]; ++nC;
            } else {                              // kept
                if (n2 >= kMaxFront) return -1;
                F2[n2] = k; dimsF[n2] = qd[k]; sxF[n2] = xstride[i]; smF[n2] = 0; ++n2;
            }
        }
        for (int l = 0; l < kMaxDeg; ++l) {
            const int k = legedge[v][l];
            if (k < 0) continue;
            const int other = ends[k][0] == v ? ends[k][1] : ends[k][0];
            if (visited[other] && other != v) continue;   // already closed above
            if (n2 >= kMaxFront) return -1;
            F2[n2] = k; dimsF[n2] = qd[k]; sxF[n2] = 0; smF[n2] = mstride[l]; ++n2;
        }
        int outsz = 1, closz = 1;
        for (int i = 0; i < n2; ++i) outsz *= dimsF[i];
        for (int i = 0; i < nC; ++i) closz *= dimsC[i];
        int *invF = smC + kMaxClose, *invC = invF + kMaxFront;
        for (int i = 0; i < n2; ++i) invF[i] = __float_as_int(1.0f / (float)dimsF[i]);
        for (int i = 0; i < nC; ++i) invC[i] = __float_as_int(1.0f / (float)dimsC[i]);
        if (outsz > maxT) return -1;
        st[0] = P.cl_verts[c * P.vwidth + v];
        st[1] = mask[v];
        st[2] = n2; st[3] = nC; st[4] = outsz; st[5] = closz;
        st[6] = v;                              // slot of the site in the cluster's vertex list
        sites_out[t] = v;
        for (int i = 0; i < n2; ++i) F[i] = F2[i];
        nF = n2;
    }
    return nv;
}

// The same plan built by a whole warp: the greedy choice of each step is
// evaluated by one lane per candidate site and settled by a warp minimum over
// (new frontier, work, slot) — the serial order of preference — and lane 0
// writes the step.  Working tables live in the warp's shared memory.
struct PlanWork {
    int legedge[kMaxSteps][kMaxDeg];
    int mask[kMaxSteps];
    int ends[32][2];
    int qd[32];
    int visited[kMaxSteps];
    int F[kMaxFront];
    int nF, fail;
};
static_assert(sizeof(PlanWork) <= 384 * sizeof(int), "plan work area");

__device__ int build_plan_warp(const ContractParams &P, int64_t c, int *plan, int *sites_out, int maxT, PlanWork &W,
                               int lane)
{
    const int32_t *E = P.cl_edges + c * P.width;
    const int32_t *V = P.cl_verts + c * P.vwidth;
    const int s = __popc(__ballot_sync(0xffffffffu, lane < P.width && E[lane] >= 0));
    const int nv = __popc(__ballot_sync(0xffffffffu, lane < P.vwidth && V[lane] >= 0)) +
                   ((P.vwidth > 32 && V[32] >= 0) ? 1 : 0);
    if (nv > kMaxSteps) return -1;
    for (int i = lane; i < kMaxSteps * kMaxDeg; i += 32) (&W.legedge[0][0])[i] = -1;
    if (lane < kMaxSteps) { W.mask[lane] = 0; W.visited[lane] = 0; }
    if (lane == 0) { W.fail = 0; W.nF = 0; }
    __syncwarp();
    if (lane < s) {
        const int k = lane, e = E[k];
        W.qd[k] = P.bond_dim[e] - 1;
        for (int side = 0; side < 2; ++side) {
            const int x = P.bond_site[2 * e + side];
            int lo = 0, hi = nv - 1, slot = -1;
            while (lo <= hi) { const int mid = (lo + hi) >> 1; if (V[mid] == x) { slot = mid; break; } if (V[mid] < x) lo = mid + 1; else hi = mid - 1; }
            if (slot < 0) { W.fail = 1; continue; }
            W.ends[k][side] = slot;
            const int leg = P.bond_leg[2 * e + side];
            W.legedge[slot][leg] = k;
            atomicOr(&W.mask[slot], 1 << leg);
        }
    }
    __syncwarp();
    if (W.fail) return -1;
    for (int t = 0; t < nv; ++t) {
        unsigned key = 0xffffffffu;
        if (lane < nv && !W.visited[lane]) {
            int closing = 0, nnew = 0;
            for (int l = 0; l < kMaxDeg; ++l) {
                const int k = W.legedge[lane][l];
                if (k < 0) continue;
                const int other = W.ends[k][0] == lane ? W.ends[k][1] : W.ends[k][0];
                if (W.visited[other]) ++closing; else ++nnew;
            }
            const int f = W.nF - closing + nnew, wk = W.nF + nnew;
            key = ((unsigned)f << 20) | ((unsigned)wk << 8) | (unsigned)lane;
        }
        key = __reduce_min_sync(0xffffffffu, key);
        const int v = (int)(key & 0xFF);
        if (lane == 0) {
            W.visited[v] = 1;
            int *st = plan + t * kStepInts;
            int *dimsF = st + 8, *sxF = dimsF + kMaxFront, *smF = sxF + kMaxFront;
            int *dimsC = smF + kMaxFront, *sxC = dimsC + kMaxClose, *smC = sxC + kMaxClose;
            int mstride[kMaxDeg];
            {
                int mul = 1;
                for (int l = kMaxDeg - 1; l >= 0; --l)
                    if (W.legedge[v][l] >= 0) { mstride[l] = mul; mul *= W.qd[W.legedge[v][l]]; }
            }
            int xstride[kMaxFront];
            {
                int mul = 1;
                for (int i = W.nF - 1; i >= 0; --i) { xstride[i] = mul; mul *= W.qd[W.F[i]]; }
            }
            int F2[kMaxFront], n2 = 0, nC = 0;
            for (int i = 0; i < W.nF && !W.fail; ++i) {
                const int k = W.F[i];
                int leg = -1;
                for (int l = 0; l < kMaxDeg; ++l) if (W.legedge[v][l] == k) leg = l;
                if (leg >= 0) {
                    dimsC[nC] = W.qd[k]; sxC[nC] = xstride[i]; smC[nC] = mstride[leg]; ++nC;
                } else if (n2 >= kMaxFront) {
                    W.fail = 1;
                } else {
                    F2[n2] = k; dimsF[n2] = W.qd[k]; sxF[n2] = xstride[i]; smF[n2] = 0; ++n2;
                }
            }
            for (int l = 0; l < kMaxDeg && !W.fail; ++l) {
                const int k = W.legedge[v][l];
                if (k < 0) continue;
                const int other = W.ends[k][0] == v ? W.ends[k][1] : W.ends[k][0];
                if (W.visited[other] && other != v) continue;   // already closed above
                if (n2 >= kMaxFront) { W.fail = 1; break; }
                F2[n2] = k; dimsF[n2] = W.qd[k]; sxF[n2] = 0; smF[n2] = mstride[l]; ++n2;
            }
            if (!W.fail) {
                int outsz = 1, closz = 1;
                for (int i = 0; i < n2; ++i) outsz *= dimsF[i];
                for (int i = 0; i < nC; ++i) closz *= dimsC[i];
                int *invF = smC + kMaxClose, *invC = invF + kMaxFront;
                for (int i = 0; i < n2; ++i) invF[i] = __float_as_int(1.0f / (float)dimsF[i]);
                for (int i = 0; i < nC; ++i) invC[i] = __float_as_int(1.0f / (float)dimsC[i]);
                if (outsz > maxT) W.fail = 1;
                st[0] = V[v];
                st[1] = W.mask[v];
                st[2] = n2; st[3] = nC; st[4] = outsz; st[5] = closz;
                st[6] = v;
                sites_out[t] = v;
                for (int i = 0; i < n2; ++i) W.F[i] = F2[i];
                W.nF = n2;
            }
        }
        __syncwarp();
        if (W.fail) return -1;
    }
    return nv;
}

template <typename T, typename L, int R>
__global__ void __launch_bounds__(kCtWarps * 32) contract_general_kernel(ContractParams P)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *plan = (int *)smem_raw + wib * (kMaxSteps * kStepInts + kMaxSteps + 4);
    int *sites = plan + kMaxSteps * kStepInts;
    int *hdr = sites + kMaxSteps;
    T *bufs = (T *)((int *)smem_raw + kCtWarps * (kMaxSteps * kStepInts + kMaxSteps + 4));
    T *X0 = bufs + (int64_t)wib * 2 * kWarpTensorMax;
    T *X1 = X0 + kWarpTensorMax;
    for (int64_t c = (int64_t)blockIdx.x * kCtWarps + wib; c < P.n_clusters; c += (int64_t)gridDim.x * kCtWarps) {
        if (lane == 0) hdr[0] = build_plan(P, c, plan, sites, kWarpTensorMax);
        __syncwarp();
        const int nsteps = hdr[0];
        if (nsteps < 0) {
            if (lane == 0) atomicExch(P.status, 1);
            for (int b = lane; b < P.n_members; b += 32) {
                P.w[(int64_t)b * P.n_clusters + c] = 0.0;
                P.nzc[(int64_t)b * P.n_clusters + c] = 0;
            }
            continue;
        }
        for (int b = 0; b < P.n_members; ++b) {
            T *X = X0, *Y = X1;
            if (lane == 0) X[0] = (T)1;
            __syncwarp();
            int expo = 0;
            for (int t = 0; t < nsteps; ++t) {
                const int *st = plan + t * kStepInts;
                const int site = st[0], mask = st[1], nF = st[2], nC = st[3], outsz = st[4], closz = st[5];
                const int *dimsF = st + 8, *sxF = dimsF + kMaxFront, *smF = sxF + kMaxFront;
                const int *dimsC = smF + kMaxFront, *sxC = dimsC + kMaxClose, *smC = sxC + kMaxClose;
            const int *invF = smC + kMaxClose, *invC = invF + kMaxFront;
                const int64_t mbase = (int64_t)b * P.stride + P.tens_off[site] + P.blk_off[site * kBlkStride + mask];
                T mx = (T)0;
                for (int o = lane; o < outsz; o += 32) {
                    int r = o, xb = 0, mb = 0;
                    for (int i = nF - 1; i >= 0; --i) { int d; r = fdivmod(r, dimsF[i], __int_as_float(invF[i]), d); xb += d * sxF[i]; mb += d * smF[i]; }
                    T acc = (T)0;
                    for (int cc = 0; cc < closz; ++cc) {
                        int rc = cc, xi = xb, mi = mb;
                        for (int i = nC - 1; i >= 0; --i) { int d; rc = fdivmod(rc, dimsC[i], __int_as_float(invC[i]), d); xi += d * sxC[i]; mi += d * smC[i]; }
                        acc = fma(rnd<R>(X[xi]), (T)L::get(P.M, mbase + mi), acc);
                    }
                    Y[o] = acc;
                    mx = fmax(mx, fabs(acc));
                }
                for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
                __syncwarp();
                if (mx > (T)0) {
                    int e;
                    frexp((double)mx, &e);
                    const T sc = (T)pow2(-e);
                    for (int o = lane; o < outsz; o += 32) Y[o] *= sc;
                    expo += e;
                }
                __syncwarp();
                T *tmp = X; X = Y; Y = tmp;
            }
            if (lane == 0) {
                double wv = ldexp((double)X[0], expo);
                int nz = 0;
                for (int t = 0; t < nsteps; ++t) {
                    const int site = plan[t * kStepInts];
                    if (P.zero[(int64_t)b * P.n_sites + site]) { ++nz; wv *= P.scale[(int64_t)b * P.n_sites + site]; }
                }
                P.w[(int64_t)b * P.n_clusters + c] = wv;
                P.nzc[(int64_t)b * P.n_clusters + c] = nz;
            }
            __syncwarp();
        }
    }
}

// Bond dimension 2: one excited value per bond, one number per site.
template <typename T, typename L>
__global__ void contract_q1_kernel(ContractParams P)
{
    const int64_t total = P.n_clusters * P.n_members;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = i % P.n_clusters;
        const int b = (int)(i / P.n_clusters);
        const int32_t *E = P.cl_edges + c * P.width;
        const int32_t *V = P.cl_verts + c * P.vwidth;
        T prod = (T)1;
        int expo = 0, nz = 0;
        double zs = 1.0;
        for (int j = 0; j < P.vwidth && V[j] >= 0; ++j) {
            const int x = V[j];
            int mask = 0;
            for (int k = 0; k < P.width && E[k] >= 0; ++k) {
                const int e = E[k];
                if (P.bond_site[2 * e] == x) mask |= 1 << P.bond_leg[2 * e];
                if (P.bond_site[2 * e + 1] == x) mask |= 1 << P.bond_leg[2 * e + 1];
            }
            const T m = (T)L::get(P.M, (int64_t)b * P.stride + P.tens_off[x] + P.blk_off[x * kBlkStride + mask]);
            prod *= m;
            if (prod != (T)0) { int e; frexp((double)prod, &e); prod *= (T)pow2(-e); expo += e; }
            if (P.zero[(int64_t)b * P.n_sites + x]) { ++nz; zs *= P.scale[(int64_t)b * P.n_sites + x]; }
        }
        P.w[(int64_t)b * P.n_clusters + c] = ldexp((double)prod, expo) * zs;
        P.nzc[(int64_t)b * P.n_clusters + c] = nz;
    }
}

// ---------------------------------------------------------------- sums
struct SumDesc {
    int32_t level;       // 0: single clusters, l >= 1: rec.levels[l-1]
    int32_t order;
    int64_t begin, end;
};

struct SumParams {
    const SumDesc *desc;
    int n_desc;
    int n_members;
    int64_t n_clusters;
    const double *w;
    const int32_t *nzc;
    const double *vac;        // [members][3]
    const int32_t *lvl_idx[16];
    int lvl_m[16];
    double *partial;          // [members][n_desc][2]
    unsigned int *done;       // [members] finished blocks (zero between calls)
    double *out;              // [members][K+1][2]
    int K;
};

constexpr int kSumThreads = 256;
constexpr int64_t kSumChunk = 4096;

__global__ void __launch_bounds__(kSumThreads) term_sum_kernel(SumParams P)
{
    __shared__ double sh[2][kSumThreads];
    const int di = blockIdx.x, b = blockIdx.y;
    const SumDesc d = P.desc[di];
    const int nzero = (int)P.vac[3 * b + 2];
    const double *w = P.w + (int64_t)b * P.n_clusters;
    const int32_t *nz = P.nzc + (int64_t)b * P.n_clusters;
    double s = 0.0, a = 0.0;
    if (d.level == 0) {
        for (int64_t i = d.begin + threadIdx.x; i < d.end; i += kSumThreads) {
            const double v = (nz[i] == nzero) ? w[i] : 0.0;
            s += v; a += fabs(v);
        }
    } else {
        const int m = P.lvl_m[d.level - 1];
        const int32_t *idx = P.lvl_idx[d.level - 1];
        for (int64_t i = d.begin + threadIdx.x; i < d.end; i += kSumThreads) {
            const int32_t *tp = idx + i * m;
            double v = 1.0;
            int z = 0;
            for (int q = 0; q < m; ++q) { v *= w[tp[q]]; z += nz[tp[q]]; }
            if (z != nzero) v = 0.0;
            s += v; a += fabs(v);
        }
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = a;
    __syncthreads();
    for (int off = kSumThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + off];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    // the member's last block to finish reduces its partials, per order in
    // descriptor order (the same sums as finalize_kernel), and re-arms the counter
    __shared__ int last;
    if (threadIdx.x == 0) {
        P.partial[((int64_t)b * P.n_desc + di) * 2] = sh[0][0];
        P.partial[((int64_t)b * P.n_desc + di) * 2 + 1] = sh[1][0];
        __threadfence();
        last = atomicAdd(P.done + b, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int k = threadIdx.x; k <= P.K; k += blockDim.x) {
        double ss = 0.0, aa = 0.0;
        for (int d2 = 0; d2 < P.n_desc; ++d2)
            if (P.desc[d2].order == k) {
                ss += __ldcg(P.partial + ((int64_t)b * P.n_desc + d2) * 2);
                aa += __ldcg(P.partial + ((int64_t)b * P.n_desc + d2) * 2 + 1);
            }
        P.out[((int64_t)b * (P.K + 1) + k) * 2] = ss;
        P.out[((int64_t)b * (P.K + 1) + k) * 2 + 1] = aa;
    }
    if (threadIdx.x == 0) P.done[b] = 0u;
}

// per (member, order): partials of that order in descriptor order
__global__ void finalize_kernel(const double *partial, const SumDesc *desc, int n_desc, int n_members, int K,
                                double *out /* [members][K+1][2] */)
{
    const int64_t total = (int64_t)n_members * (K + 1);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(i / (K + 1)), k = (int)(i % (K + 1));
        double s = 0.0, a = 0.0;
        for (int d = 0; d < n_desc; ++d)
            if (desc[d].order == k) {
                s += partial[((int64_t)b * n_desc + d) * 2];
                a += partial[((int64_t)b * n_desc + d) * 2 + 1];
            }
        out[i * 2] = s;
        out[i * 2 + 1] = a;
    }
}

// ---------------------------------------------------------------- ALL mode
// Every subset E of the closed bonds (at most 30) with |E| <= K is a term.
// Subsets of size k are visited by unranking k-combinations (colexicographic
// order of the combinatorial number system).  Bond dimension 2 only: the term
// divided by the vacuum is prod_v M_v[excited legs of v] over touched sites.
struct AllParams {
    int n_members, n_sites, Mc, K;
    const int32_t *site_ptr, *site_bonds;  // closed geometry
    const int32_t *blk_off;
    const int64_t *tens_off;
    int64_t stride;
    const void *M;
    const double *scale;
    const int8_t *zero;
    const double *vac;
    const int64_t *binom;                  // [31][31]
    const SumDesc *desc;                   // order, rank range [begin, end)
    int n_desc;
    double *partial;                       // [members][n_desc][2]
    int64_t *conn_count;                   // [n_desc]: connected subsets (member 0 only)
    const int32_t *bond_site;
};

__device__ uint32_t unrank_comb(int64_t r, int k, const int64_t *binom)
{
    uint32_t mask = 0;
    for (int i = k; i >= 1; --i) {
        int c = i - 1;
        while (binom[(c + 1) * 31 + i] <= r) ++c;
        r -= binom[c * 31 + i];
        mask |= 1u << c;
    }
    return mask;
}

template <typename T, typename L>
__global__ void __launch_bounds__(kSumThreads) all_q1_kernel(AllParams P)
{
    __shared__ double sh[2][kSumThreads];
    __shared__ long long shc[kSumThreads];
    const int di = blockIdx.x, b = blockIdx.y;
    const SumDesc d = P.desc[di];
    const int nzero = (int)P.vac[3 * b + 2];
    double s = 0.0, a = 0.0;
    long long conn = 0;
    for (int64_t r = d.begin + threadIdx.x; r < d.end; r += kSumThreads) {
        const uint32_t E = unrank_comb(r, d.order, P.binom);
        T prod = (T)1;
        int expo = 0, cover = 0;
        double zs = 1.0;
        for (int v = 0; v < P.n_sites; ++v) {
            int mask = 0;
            for (int p = P.site_ptr[v]; p < P.site_ptr[v + 1]; ++p)
                if ((E >> P.site_bonds[p]) & 1u) mask |= 1 << (p - P.site_ptr[v]);
            if (mask == 0) continue;
            prod *= (T)L::get(P.M, (int64_t)b * P.stride + P.tens_off[v] + P.blk_off[v * kBlkStride + mask]);
            if (prod != (T)0) { int e; frexp((double)prod, &e); prod *= (T)pow2(-e); expo += e; }
            if (P.zero[(int64_t)b * P.n_sites + v]) { ++cover; zs *= P.scale[(int64_t)b * P.n_sites + v]; }
        }
        double val = (cover == nzero) ? ldexp((double)prod, expo) * zs : 0.0;
        if (d.order == 0) val = (nzero == 0) ? 1.0 : 0.0;
        s += val; a += fabs(val);
        if (b == 0 && E != 0) {
            // connectivity of E by vertex-set growth
            uint32_t left = E & ~(E & (0u - E));
            uint64_t cov = 0;
            {
                const int e0 = __ffs(E) - 1;
                cov = (1ull << P.bond_site[2 * e0]) | (1ull << P.bond_site[2 * e0 + 1]);
            }
            bool grew = true;
            while (grew && left) {
                grew = false;
                for (uint32_t rr = left; rr; rr &= rr - 1) {
                    const int e = __ffs(rr) - 1;
                    const uint64_t vm = (1ull << P.bond_site[2 * e]) | (1ull << P.bond_site[2 * e + 1]);
                    if (vm & cov) { cov |= vm; left &= ~(1u << e); grew = true; }
                }
            }
            if (!left) ++conn;
        }
    }
    sh[0][threadIdx.x] = s; sh[1][threadIdx.x] = a; shc[threadIdx.x] = conn;
    __syncthreads();
    for (int off = kSumThreads / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + off];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + off];
            shc[threadIdx.x] += shc[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        P.partial[((int64_t)b * P.n_desc + di) * 2] = sh[0][0];
        P.partial[((int64_t)b * P.n_desc + di) * 2 + 1] = sh[1][0];
        if (b == 0) P.conn_count[di] = shc[0];
    }
}

int grid_for(int64_t n, int block, int n_sm, int per_sm = 32)
{
    int64_t g = (n + block - 1) / block;
    const int64_t cap = (int64_t)n_sm * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

bool all_dims_two(const Geometry &g)
{
    for (int b = 0; b < g.n_bonds; ++b) if (g.bond_dim[b] != 2) return false;
    return true;
}

template <typename KERN>
pne_status run_general(pne_ctx *ctx, KERN kern, const ContractParams &cp, size_t elem, cudaStream_t s)
{
    const size_t smem = (size_t)kCtWarps * ((kMaxSteps * kStepInts + kMaxSteps + 4) * 4 + 2 * kWarpTensorMax * elem);
    grant_dynamic_smem((const void *)kern, smem);
    const int g = grid_for(cp.n_clusters, kCtWarps, ctx->n_sm, 16);
    kern<<<g, kCtWarps * 32, smem, s>>>(cp);
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}

}  // namespace

namespace {

constexpr int kPlanInts = kMaxSteps * kStepInts;
constexpr int kClassMin = 8;           // smallest running-tensor class of the shaped contraction
// shared ints per warp of the plan kernel: plan, sites, spare, then a PlanWork
// (declared below; its size is checked there)
constexpr int kPlanWarpInts = kMaxSteps * kStepInts + kMaxSteps + 4 + 384;

// Local structure of a cluster, independent of where it sits: site slots
// (rank in the sorted vertex list), the leg of each bond end and each bond's
// excited dimension.  Clusters with equal keys have equal plans.
__device__ int cluster_key(const ContractParams &P, int64_t c, int32_t *key, int cap)
{
    const int32_t *E = P.cl_edges + c * P.width;
    const int32_t *V = P.cl_verts + c * P.vwidth;
    int s = 0, nv = 0;
    while (s < P.width && E[s] >= 0) ++s;
    while (nv < P.vwidth && V[nv] >= 0) ++nv;
    int n = 0;
    key[n++] = nv; key[n++] = s;
    for (int k = 0; k < s && n + 5 <= cap; ++k) {
        const int e = E[k];
        for (int side = 0; side < 2; ++side) {
            const int x = P.bond_site[2 * e + side];
            int slot = 0;
            while (slot < nv && V[slot] != x) ++slot;
            key[n++] = slot;
            key[n++] = P.bond_leg[2 * e + side];
        }
        key[n++] = P.bond_dim[e];
    }
    return n;
}

__global__ void shape_hash_kernel(ContractParams P, unsigned long long *hash)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < P.n_clusters;
         c += (int64_t)gridDim.x * blockDim.x) {
        int32_t key[2 + 5 * 32];
        const int n = cluster_key(P, c, key, 2 + 5 * 32);
        unsigned long long h = 1469598103934665603ull;
        for (int i = 0; i < n; ++i) {
            h ^= (unsigned long long)(uint32_t)key[i];
            h *= 1099511628211ull;
            h ^= h >> 29;
        }
        hash[c] = h;
    }
}

// 1 where a cluster's key differs from its shape representative's (a hash collision)
__device__ void verify_range(const ContractParams &P, const int32_t *shape_of, const int32_t *rep, int32_t *bad,
                             int64_t first, int64_t stride)
{
    for (int64_t c = first; c < P.n_clusters; c += stride) {
        int32_t a[2 + 5 * 32], b[2 + 5 * 32];
        const int na = cluster_key(P, c, a, 2 + 5 * 32);
        const int nb = cluster_key(P, rep[shape_of[c]], b, 2 + 5 * 32);
        int d = (na != nb);
        for (int i = 0; i < na && !d; ++i) d = (a[i] != b[i]);
        bad[c] = d;
    }
}

// One plan per shape (built by lane 0 of a warp), plus the per-shape figures the
// host needs: stats[sh] = {steps (-1: no plan), multiply-adds, largest running
// tensor, 0}.
__device__ void plan_range(const ContractParams &P, const int32_t *rep, int n_shapes, int32_t *plans, int32_t *steps,
                           int32_t *stats, int bid, int nblk)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *plan = (int *)smem_raw + wib * kPlanWarpInts;
    int *sites = plan + kMaxSteps * kStepInts;
    PlanWork &W = *reinterpret_cast<PlanWork *>(sites + kMaxSteps + 4);
    for (int sh = bid * kCtWarps + wib; sh < n_shapes; sh += nblk * kCtWarps) {
        const int n = build_plan_warp(P, rep[sh], plan, sites, kWarpTensorMax, W, lane);
        if (lane == 0) {
            steps[sh] = n;
            int fma = 0, mo = 1;
            for (int t = 0; t < n; ++t) { fma += plan[t * kStepInts + 4] * plan[t * kStepInts + 5]; mo = max(mo, plan[t * kStepInts + 4]); }
            stats[4 * sh] = n; stats[4 * sh + 1] = fma; stats[4 * sh + 2] = mo; stats[4 * sh + 3] = 0;
        }
        __syncwarp();
        for (int i = lane; i < (n > 0 ? n : 0) * kStepInts; i += 32) plans[(int64_t)sh * kPlanInts + i] = plan[i];
        __syncwarp();
    }
}

__global__ void shape_plan_kernel(ContractParams P, const int32_t *rep, int n_shapes, int32_t *plans,
                                  int32_t *steps, int32_t *stats)
{
    plan_range(P, rep, n_shapes, plans, steps, stats, blockIdx.x, gridDim.x);
}

// The exact-key check of every cluster against its representative and the
// representatives' plans in one launch: blocks [0, plan_blocks) build plans,
// the others check keys (one thread per cluster), so the two run side by side.
__global__ void shape_verify_plan_kernel(ContractParams P, const int32_t *shape_of, const int32_t *rep, int32_t *bad,
                                         int n_shapes, int32_t *plans, int32_t *steps, int32_t *stats, int plan_blocks)
{
    if ((int)blockIdx.x < plan_blocks) {
        plan_range(P, rep, n_shapes, plans, steps, stats, blockIdx.x, plan_blocks);
    } else {
        const int64_t vb = (int64_t)blockIdx.x - plan_blocks, nvb = (int64_t)gridDim.x - plan_blocks;
        verify_range(P, shape_of, rep, bad, vb * blockDim.x + threadIdx.x, nvb * blockDim.x);
    }
}

// The multiply-adds of every step of a shape's plan, in the order the
// contraction runs them (step, output entry o, closed entry cc), each packed as
// (xi << 16) | mi: xi indexes the running tensor, mi the site's excited block.
// One warp per shape; the plan's digit decoding is done here once instead of
// per cluster and per multiply-add.
__global__ void shape_ops_kernel(const int32_t *plans, const int32_t *plan_steps, const int64_t *op_off, int n_shapes,
                                 int32_t *ops)
{
    const int lane = threadIdx.x & 31;
    for (int sh = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sh < n_shapes; sh += (gridDim.x * blockDim.x) >> 5) {
        const int *plan = plans + (int64_t)sh * kPlanInts;
        int64_t at = op_off[sh];
        for (int t = 0; t < plan_steps[sh]; ++t) {
            const int *st = plan + t * kStepInts;
            const int nF = st[2], nC = st[3], outsz = st[4], closz = st[5];
            const int *dimsF = st + 8, *sxF = dimsF + kMaxFront, *smF = sxF + kMaxFront;
            const int *dimsC = smF + kMaxFront, *sxC = dimsC + kMaxClose, *smC = sxC + kMaxClose;
            for (int idx = lane; idx < outsz * closz; idx += 32) {
                int r = idx / closz, rc = idx % closz, xi = 0, mi = 0;
                for (int q = nF - 1; q >= 0; --q) { const int d = r % dimsF[q]; r /= dimsF[q]; xi += d * sxF[q]; mi += d * smF[q]; }
                for (int q = nC - 1; q >= 0; --q) { const int d = rc % dimsC[q]; rc /= dimsC[q]; xi += d * sxC[q]; mi += d * smC[q]; }
                // xi < 256 (shaped plans keep every running tensor within 256
                // entries) and mi < 4096 (site tensors hold at most 4096 entries)
                ops[at + idx] = (xi << 16) | mi;
            }
            at += (int64_t)outsz * closz;
        }
    }
}

// Per cluster and plan step: the site and the offset of its excited block
// within one tensor set (geometry only), so that the contraction reads each
// step's block base with one independent load.
__global__ void cluster_steps_kernel(ContractParams P, const int32_t *shape_of, const int32_t *plans,
                                     const int32_t *plan_steps, int stride, int32_t *step_off, int32_t *step_site)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < P.n_clusters;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int sh = shape_of[c];
        const int *plan = plans + (int64_t)sh * kPlanInts;
        const int32_t *V = P.cl_verts + c * P.vwidth;
        for (int t = 0; t < plan_steps[sh]; ++t) {
            const int site = V[plan[t * kStepInts + 6]];
            step_site[c * stride + t] = site;
            step_off[c * stride + t] = (int32_t)(P.tens_off[site] + P.blk_off[site * kBlkStride + plan[t * kStepInts + 1]]);
        }
    }
}

// Exponent handling of the running tensor on the integer pipes: the biased
// exponent of a value, and 2^-e built from bits.  Rescaling by a power of two is
// exact, so when it happens does not change a single bit of the result (short of
// overflow or subnormals): FP64 rescales only when the largest entry leaves
// 2^[-64, 64], the FP32 family after every step.
template <typename T> struct Expo;
template <> struct Expo<double> {
    static constexpr int kBias = 1023, kWindow = 64;
    __device__ static int biased(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }
    __device__ static double inv_pow2(int e) { return __longlong_as_double((long long)(kBias - e) << 52); }   // e < kBias
};
template <> struct Expo<float> {
    static constexpr int kBias = 127, kWindow = 0;
    __device__ static int biased(float x) { return (__float_as_int(x) >> 23) & 0xFF; }
    __device__ static float inv_pow2(int e) { return __int_as_float((kBias - e) << 23); }   // e < kBias
};

// One cluster c of tensor set b by its shape's plan.  The lane keeps its
// running tensor at X[j * 32] (interleaved with the other lanes, so shared
// memory is conflict-free).  Each output entry is a chain of fused
// multiply-adds in the plan's order; the multiply-add list is walked eight at a
// time with all loads of a group issued before its chain, so the latency of
// the site-tensor loads overlaps.  Every contraction path (one network, the
// fused batch) runs this routine, so their values agree bit for bit.
template <typename T, typename L, int R>
__device__ __forceinline__ void shaped_cluster(const ContractParams &P, const int *plan, int nsteps, const int32_t *ops,
                                               const int32_t *soff, const int32_t *ssite, int64_t c, int b, T *X, T *Y)
{
    X[0] = (T)1;
    int expo = 0, nz = 0;
    double zs = 1.0;
    for (int t = 0; t < nsteps; ++t) {
        const int *st = plan + t * kStepInts;
        const int outsz = st[4], closz = st[5];
        const int64_t mbase = (int64_t)b * P.stride + __ldg(soff + t);
        int mxb = 0;                                   // largest biased exponent among the outputs
        // the step's (o, cc) list walked flat, eight multiply-adds at a time:
        // a group's loads are issued together even when it spans outputs
        const int n_ops = outsz * closz;
        T acc = (T)0;
        int cc = 0, o = 0;
        for (int k0 = 0; k0 < n_ops; k0 += 8) {
            const int m = min(8, n_ops - k0);
            int32_t pk[8];
            T xv[8], mv[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) pk[k] = (k < m) ? __ldg(ops + k0 + k) : 0;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                xv[k] = rnd<R>(X[(pk[k] >> 16) * 32]);
                mv[k] = (k < m) ? (T)L::get(P.M, mbase + (pk[k] & 0xffff)) : (T)0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k < m) {
                    acc = fma(xv[k], mv[k], acc);
                    if (++cc == closz) {
                        Y[o * 32] = acc;
                        mxb = max(mxb, Expo<T>::biased(acc));
                        acc = (T)0; cc = 0; ++o;
                    }
                }
            }
        }
        ops += n_ops;
        if (mxb > 0) {
            const int e = mxb - (Expo<T>::kBias - 1);      // the frexp exponent of the largest entry
            if (e > Expo<T>::kWindow || e < -Expo<T>::kWindow) {
                const T sc = (e < Expo<T>::kBias) ? Expo<T>::inv_pow2(e) : (T)ldexp(1.0, -e);   // 2^-e
                for (int o = 0; o < outsz; ++o) Y[o * 32] *= sc;
                expo += e;
            }
        }
        T *tmp = X; X = Y; Y = tmp;
        const int site = __ldg(ssite + t);
        if (P.zero[(int64_t)b * P.n_sites + site]) { ++nz; zs *= P.scale[(int64_t)b * P.n_sites + site]; }
    }
    P.w[(int64_t)b * P.n_clusters + c] = ldexp((double)X[0], expo) * zs;
    P.nzc[(int64_t)b * P.n_clusters + c] = nz;
}

// Side streams of the context, created on first use (caller holds side_mu).
pne_status side_streams(pne_ctx *ctx)
{
    if (ctx->side_ready) return PNE_OK;
    for (auto &st : ctx->side) PNE_CUDA_TRY(ctx, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    for (auto &ev : ctx->side_ev) PNE_CUDA_TRY(ctx, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ctx->side_ready = true;
    return PNE_OK;
}

// One cluster c of tensor set b contracted by a group of G lanes (lane `sub`
// of the group, mask `gmask`): the running tensor X/Y sits once in shared
// memory and the group's lanes split each step's outputs (lane j takes
// outputs j, j + G, ...).  Every output is the same chain of multiply-adds in
// the same order as in shaped_cluster, and the rescaling decision is the same,
// so the values agree bit for bit with the lane-per-cluster form.
template <typename T, typename L, int R, int G>
__device__ __forceinline__ void group_cluster(const ContractParams &P, const int *plan, int nsteps, const int32_t *op,
                                              const int32_t *soff, const int32_t *ssite, int64_t c, int b, T *X, T *Y,
                                              int sub, unsigned gmask)
{
    if (sub == 0) X[0] = (T)1;
    __syncwarp(gmask);
    int expo = 0, nz = 0;
    double zs = 1.0;
    for (int t = 0; t < nsteps; ++t) {
        const int *st = plan + t * kStepInts;
        const int outsz = st[4], closz = st[5];
        const int64_t mbase = (int64_t)b * P.stride + __ldg(soff + t);
        int mxb = 0;
        for (int o = sub; o < outsz; o += G) {
            const int32_t *oo = op + (int64_t)o * closz;
            T acc = (T)0;
            int cc = 0;
            for (; cc + 4 <= closz; cc += 4) {
                int32_t pk[4];
                T xv[4], mv[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) pk[k] = __ldg(oo + cc + k);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    xv[k] = rnd<R>(X[pk[k] >> 16]);
                    mv[k] = (T)L::get(P.M, mbase + (pk[k] & 0xffff));
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) acc = fma(xv[k], mv[k], acc);
            }
            for (; cc < closz; ++cc) {
                const int32_t pk = __ldg(oo + cc);
                acc = fma(rnd<R>(X[pk >> 16]), (T)L::get(P.M, mbase + (pk & 0xffff)), acc);
            }
            Y[o] = acc;
            mxb = max(mxb, Expo<T>::biased(acc));
        }
        op += (int64_t)outsz * closz;
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) mxb = max(mxb, __shfl_xor_sync(gmask, mxb, off));
        __syncwarp(gmask);
        if (mxb > 0) {
            const int e = mxb - (Expo<T>::kBias - 1);
            if (e > Expo<T>::kWindow || e < -Expo<T>::kWindow) {
                const T sc = (e < Expo<T>::kBias) ? Expo<T>::inv_pow2(e) : (T)ldexp(1.0, -e);
                for (int o = sub; o < outsz; o += G) Y[o] *= sc;
                expo += e;
                __syncwarp(gmask);
            }
        }
        T *tmp = X; X = Y; Y = tmp;
        const int site = __ldg(ssite + t);
        if (P.zero[(int64_t)b * P.n_sites + site]) { ++nz; zs *= P.scale[(int64_t)b * P.n_sites + site]; }
    }
    if (sub == 0) {
        P.w[(int64_t)b * P.n_clusters + c] = ldexp((double)X[0], expo) * zs;
        P.nzc[(int64_t)b * P.n_clusters + c] = nz;
    }
    __syncwarp(gmask);
}

template <int G>
__device__ __forceinline__ unsigned group_mask(int lane)
{
    return (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane - lane % G));
}

// Clusters perm[i0, i1) of every tensor set, a group of G lanes per (cluster,
// set) (group_cluster).  Neighbouring outputs read neighbouring block entries,
// so a warp's gathers touch 32 / G clusters instead of 32; groups sync and
// reduce over their own lane mask, so groups of different shapes in one warp
// never wait for each other.
template <typename T, typename L, int R, int G>
__global__ void __launch_bounds__(256) contract_group_kernel(ContractParams P, const int32_t *perm,
                                                             const int32_t *shape_of, const int32_t *plans,
                                                             const int32_t *plan_steps, const int32_t *ops,
                                                             const int64_t *op_off, const int32_t *step_off,
                                                             const int32_t *step_site, int sstride, int xmax,
                                                             int64_t i0, int64_t i1)
{
    static_assert(G == 4 || G == 8 || G == 16 || G == 32, "group size");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, sub = lane % G;
    const int gib = threadIdx.x / G, gpb = blockDim.x / G;            // group in block, groups per block
    const unsigned gmask = group_mask<G>(lane);
    T *X0 = (T *)smem_raw + (int64_t)gib * 2 * xmax;
    T *X1 = X0 + xmax;
    const int64_t nc = i1 - i0;
    const int64_t items = nc * P.n_members;
    for (int64_t it = (int64_t)blockIdx.x * gpb + gib; it < items; it += (int64_t)gridDim.x * gpb) {
        const int b = (int)(it / nc);
        const int64_t c = perm[i0 + it % nc];
        const int sh = shape_of[c];
        group_cluster<T, L, R, G>(P, plans + (int64_t)sh * kPlanInts, plan_steps[sh], ops + op_off[sh],
                                  step_off + c * sstride, step_site + c * sstride, c, b, X0, X1, sub, gmask);
    }
}

template <typename T, typename L, int R>
pne_status run_shaped(pne_ctx *ctx, const ContractParams &cp, const EnumRecord &rec, cudaStream_t s)
{
    // one launch per running-tensor class, each with buffers (and so an
    // occupancy) sized for its own class; the classes are independent, so
    // when there are several they run concurrently on side streams forked
    // from and joined back into `s`
    std::vector<size_t> cls;
    for (size_t q = 0; q + 1 < rec.class_start.size(); ++q)
        if (rec.class_start[q + 1] > rec.class_start[q]) cls.push_back(q);
    std::unique_lock<std::mutex> lk(ctx->side_mu, std::defer_lock);
    const bool fork = cls.size() > 1;
    if (fork) {
        lk.lock();
        pne_status st = side_streams(ctx);
        if (st) return st;
        PNE_CUDA_TRY(ctx, cudaEventRecord(ctx->side_ev[0], s));
    }
    // the largest running tensors (fewest, longest clusters) start first, on `s`
    std::reverse(cls.begin(), cls.end());
    for (size_t j = 0; j < cls.size(); ++j) {
        const size_t q = cls[j];
        const int64_t i0 = rec.class_start[q], i1 = rec.class_start[q + 1];
        const int xmax = std::min(rec.class_xmax[q], std::max(rec.max_out, 1));
        cudaStream_t ls = s;
        if (fork && j > 0) {
            ls = ctx->side[(j - 1) % pne_ctx::kSideStreams];
            PNE_CUDA_TRY(ctx, cudaStreamWaitEvent(ls, ctx->side_ev[0], 0));
        }
        {
            // a group of lanes per cluster: 32 for large running tensors, else 4
            // (8 lanes for the 16-entry class measured 89 against 78 us on
            // the 16x16 D = 4 step: fewer lanes per cluster keep more clusters'
            // gathers in flight)
            const int G = xmax >= 32 ? 32 : 4;
            const int gpb = 256 / G;
            const size_t smem2 = (size_t)gpb * 2 * xmax * sizeof(T);
            const int64_t items2 = (i1 - i0) * cp.n_members;
            int64_t g2 = (items2 + gpb - 1) / gpb;
            if (g2 > (int64_t)ctx->n_sm * 16) g2 = (int64_t)ctx->n_sm * 16;
            auto launch = [&](auto kernel) {
                grant_dynamic_smem((const void *)kernel, smem2);
                kernel<<<(int)g2, 256, smem2, ls>>>(cp, (const int32_t *)rec.perm.ptr, (const int32_t *)rec.shape_of.ptr,
                                                    (const int32_t *)rec.plans.ptr, (const int32_t *)rec.plan_steps.ptr,
                                                    (const int32_t *)rec.ops.ptr, (const int64_t *)rec.op_off.ptr,
                                                    (const int32_t *)rec.step_off.ptr, (const int32_t *)rec.step_site.ptr,
                                                    rec.step_stride, xmax, i0, i1);
            };
            if (G == 32) launch(contract_group_kernel<T, L, R, 32>);
            else if (G == 8) launch(contract_group_kernel<T, L, R, 8>);
            else launch(contract_group_kernel<T, L, R, 4>);
            PNE_CUDA_TRY(ctx, cudaGetLastError());
        }
    }
    if (fork) {
        const size_t used = std::min<size_t>(cls.size() - 1, pne_ctx::kSideStreams);
        for (size_t k = 0; k < used; ++k) {
            PNE_CUDA_TRY(ctx, cudaEventRecord(ctx->side_ev[1 + k], ctx->side[k]));
            PNE_CUDA_TRY(ctx, cudaStreamWaitEvent(s, ctx->side_ev[1 + k], 0));
        }
    }
    return PNE_OK;
}

template <typename T, typename L, int R>
pne_status dispatch_shaped(pne_ctx *ctx, const ContractParams &cp, const EnumRecord &rec, cudaStream_t s)
{
    return run_shaped<T, L, R>(ctx, cp, rec, s);
}

}  // namespace

// Shape preparation, first half: hash every cluster's local structure and
// queue the hashes' readback (no synchronisation; the caller's next
// synchronisation of `s` brings them).
bool shapes_needed(const Geometry &g, const EnumRecord &rec)
{
    return rec.n_clusters > 0 && !all_dims_two(g);
}

pne_status shapes_begin(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s)
{
    rec.shaped = false;
    sp.active = false;
    if (!shapes_needed(g, rec)) return PNE_OK;
    const int64_t n = (int64_t)rec.n_clusters;
    ContractParams cp;
    cp.n_clusters = n; cp.n_members = 1; cp.n_sites = g.n_sites;
    cp.width = rec.width; cp.vwidth = rec.vwidth;
    cp.cl_edges = (const int32_t *)rec.cl_edges.ptr; cp.cl_verts = (const int32_t *)rec.cl_verts.ptr;
    cp.cl_size = (const int32_t *)rec.cl_size.ptr;
    cp.bond_site = g.d_bond_site; cp.bond_dim = g.d_bond_dim; cp.bond_leg = g.d_bond_leg;
    pne_status st = dev_alloc(ctx, sp.dh, n * 8, s);
    if (st) return st;
    {
        ProfScope ps(ctx, s, "shapes");
        shape_hash_kernel<<<grid_for(n, 128, ctx->n_sm), 128, 0, s>>>(cp, (unsigned long long *)sp.dh.ptr);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    sp.h_pinned = pinned_slot(3, n * 8);
    if (sp.h_pinned) PNE_CUDA_TRY(ctx, cudaMemcpyAsync(sp.h_pinned, sp.dh.ptr, n * 8, cudaMemcpyDeviceToHost, s));
    sp.active = true;
    return PNE_OK;
}

namespace {

ContractParams shape_params(const Geometry &g, const EnumRecord &rec)
{
    ContractParams cp;
    cp.n_clusters = (int64_t)rec.n_clusters; cp.n_members = 1; cp.n_sites = g.n_sites;
    cp.width = rec.width; cp.vwidth = rec.vwidth;
    cp.cl_edges = (const int32_t *)rec.cl_edges.ptr; cp.cl_verts = (const int32_t *)rec.cl_verts.ptr;
    cp.cl_size = (const int32_t *)rec.cl_size.ptr;
    cp.bond_site = g.d_bond_site; cp.bond_dim = g.d_bond_dim; cp.bond_leg = g.d_bond_leg;
    return cp;
}

// One plan per representative, its statistics [steps, multiply-adds, largest
// output, 0] (and, with_bad, the verification flags) read back into pinned
// memory -- queued, or read at once when no pinned memory is available.
pne_status plans_launch(pne_ctx *ctx, const ContractParams &cp, EnumRecord &rec, ShapePrep &sp, bool with_bad,
                        cudaStream_t s)
{
    const int64_t n = cp.n_clusters;
    const int ns = sp.ns;
    dev_free(ctx, rec.plans, s);
    dev_free(ctx, rec.plan_steps, s);
    dev_free(ctx, sp.dstats, s);
    pne_status e;
    if ((e = dev_alloc(ctx, rec.plans, (size_t)ns * kPlanInts * 4, s)) ||
        (e = dev_alloc(ctx, rec.plan_steps, (size_t)ns * 4, s)) || (e = dev_alloc(ctx, sp.dstats, (size_t)ns * 16, s)))
        return e;
    const size_t smem = (size_t)kCtWarps * kPlanWarpInts * 4;
    const int pblocks = grid_for(ns, kCtWarps, ctx->n_sm, 16);
    if (with_bad) {
        // with the verification of every cluster in the same launch
        const int vblocks = grid_for(n, kCtWarps * 32, ctx->n_sm);
        shape_verify_plan_kernel<<<pblocks + vblocks, kCtWarps * 32, smem, s>>>(
            cp, (const int32_t *)sp.dshape.ptr, (const int32_t *)sp.drep.ptr, (int32_t *)sp.dbad.ptr, ns,
            (int32_t *)rec.plans.ptr, (int32_t *)rec.plan_steps.ptr, (int32_t *)sp.dstats.ptr, pblocks);
    } else {
        shape_plan_kernel<<<pblocks, kCtWarps * 32, smem, s>>>(
            cp, (const int32_t *)sp.drep.ptr, ns, (int32_t *)rec.plans.ptr, (int32_t *)rec.plan_steps.ptr,
            (int32_t *)sp.dstats.ptr);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    sp.stats.assign((size_t)ns * 4, 0);
    sp.nb = with_bad ? (size_t)n * 4 : 0;
    const size_t sb = sp.stats.size() * 4;
    sp.hp = (char *)pinned_slot(3, sp.nb + sb);
    if (sp.hp) {
        if (sp.nb) PNE_CUDA_TRY(ctx, cudaMemcpyAsync(sp.hp, sp.dbad.ptr, sp.nb, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(sp.hp + sp.nb, sp.dstats.ptr, sb, cudaMemcpyDeviceToHost, s));
    } else {
        if (sp.nb) PNE_CUDA_TRY(ctx, cudaMemcpyAsync(sp.bad.data(), sp.dbad.ptr, sp.nb, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(sp.stats.data(), sp.dstats.ptr, sb, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    return PNE_OK;
}

pne_status plans_read(pne_ctx *ctx, ShapePrep &sp, cudaStream_t s)
{
    if (!sp.hp) return PNE_OK;
    {
        HostScope hw__(ctx, "sync_plans");
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    if (sp.nb) std::memcpy(sp.bad.data(), sp.hp, sp.nb);
    std::memcpy(sp.stats.data(), sp.hp + sp.nb, sp.stats.size() * 4);
    sp.hp = nullptr;
    return PNE_OK;
}

}  // namespace

void shapes_release(pne_ctx *ctx, ShapePrep &sp, cudaStream_t s)
{
    dev_free(ctx, sp.dh, s);
    dev_free(ctx, sp.dshape, s);
    dev_free(ctx, sp.drep, s);
    dev_free(ctx, sp.dbad, s);
    dev_free(ctx, sp.dstats, s);
    sp.active = sp.planned = false;
}

// Second stage: shape ids in order of first appearance (deterministic), an
// exact-key check of every cluster against its representative, one plan per
// representative; the flags and plan statistics are read back by
// shapes_complete.
pne_status shapes_plan(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s)
{
    if (!sp.active) return PNE_OK;
    sp.active = false;
    const int64_t n = (int64_t)rec.n_clusters;
    const ContractParams cp = shape_params(g, rec);
    pne_status st;
    std::vector<unsigned long long> hv;
    const unsigned long long *h = (const unsigned long long *)sp.h_pinned;
    if (sp.h_pinned) {
        HostScope hw__(ctx, "sync_shapes");
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    } else {
        hv.resize(n);
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(hv.data(), sp.dh.ptr, n * 8, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        h = hv.data();
    }
    dev_free(ctx, sp.dh, s);
    // shape ids by first appearance: an open-addressing table of the hashes
    // (linear probing, at most half full)
    size_t cap = 64;
    while (cap < 2 * (size_t)n) cap *= 2;
    std::vector<unsigned long long> keys(cap);
    std::vector<int32_t> vals(cap, -1);
    sp.shape.assign(n, 0);
    sp.rep.clear();
    for (int64_t c = 0; c < n; ++c) {
        const unsigned long long k = h[c];
        size_t at = (size_t)((k ^ (k >> 29)) * 0x9E3779B97F4A7C15ull) & (cap - 1);
        while (vals[at] >= 0 && keys[at] != k) at = (at + 1) & (cap - 1);
        if (vals[at] < 0) { keys[at] = k; vals[at] = (int32_t)sp.rep.size(); sp.rep.push_back((int32_t)c); }
        sp.shape[c] = vals[at];
    }
    // exact key check against the representative (a mismatch gets its own
    // shape) and the plans of the representatives, read back together
    if ((st = dev_alloc(ctx, sp.dshape, n * 4, s)) || (st = dev_alloc(ctx, sp.drep, sp.rep.size() * 4, s)) ||
        (st = dev_alloc(ctx, sp.dbad, n * 4, s)))
        return st;
    if ((st = upload(ctx, sp.dshape.ptr, sp.shape.data(), n * 4, s)) ||
        (st = upload(ctx, sp.drep.ptr, sp.rep.data(), sp.rep.size() * 4, s)))
        return st;
    sp.ns = (int)sp.rep.size();
    sp.bad.assign(n, 0);
    if ((st = plans_launch(ctx, cp, rec, sp, true, s))) return st;
    sp.planned = true;
    return PNE_OK;
}

// Third stage: the plan statistics, then the multiply-add lists of every
// shape, the clusters ordered by running-tensor class and shape, and the
// per-cluster step tables.
pne_status shapes_complete(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s)
{
    if (!sp.planned) return PNE_OK;
    sp.planned = false;
    const int64_t n = (int64_t)rec.n_clusters;
    const ContractParams cp = shape_params(g, rec);
    pne_status st;
    if ((st = plans_read(ctx, sp, s))) return st;
    std::vector<int32_t> &shape = sp.shape, &rep = sp.rep, &stats = sp.stats;
    bool any_bad = false;
    for (int64_t c = 0; c < n; ++c)
        if (sp.bad[c]) { shape[c] = (int32_t)rep.size(); rep.push_back((int32_t)c); any_bad = true; }
    if (any_bad) {
        // hash collisions (rare): the split-off clusters become representatives
        sp.ns = (int)rep.size();
        dev_free(ctx, sp.drep, s);
        if ((st = dev_alloc(ctx, sp.drep, sp.ns * 4, s))) return st;
        if ((st = upload(ctx, sp.drep.ptr, rep.data(), sp.ns * 4, s)) ||
            (st = upload(ctx, sp.dshape.ptr, shape.data(), n * 4, s)))
            return st;
        if ((st = plans_launch(ctx, cp, rec, sp, false, s)) || (st = plans_read(ctx, sp, s))) return st;
    }
    const int ns = sp.ns;
    rec.shape_fma.assign(ns, 0);
    rec.shape_count.assign(ns, 0);
    int max_out = 1;
    bool ok = true;
    std::vector<int> shape_cls(ns, 0);
    for (int i = 0; i < ns; ++i) {
        if (stats[4 * i] < 0) { ok = false; break; }
        rec.shape_fma[i] = (uint64_t)stats[4 * i + 1];
        const int mo = std::max(1, stats[4 * i + 2]);
        max_out = std::max(max_out, mo);
        while ((kClassMin << shape_cls[i]) < mo) ++shape_cls[i];
    }
    // the multiply-add lists of every shape
    if (ok) {
        std::vector<int64_t> off(ns + 1, 0);
        for (int i = 0; i < ns; ++i) off[i + 1] = off[i] + (int64_t)rec.shape_fma[i];
        dev_free(ctx, rec.ops, s);
        dev_free(ctx, rec.op_off, s);
        if ((st = dev_alloc(ctx, rec.ops, (size_t)std::max<int64_t>(off[ns], 1) * 4, s)) ||
            (st = dev_alloc(ctx, rec.op_off, (size_t)(ns + 1) * 8, s)) ||
            (st = upload(ctx, rec.op_off.ptr, off.data(), (size_t)(ns + 1) * 8, s)))
            return st;
        shape_ops_kernel<<<grid_for((int64_t)ns * 32, 128, ctx->n_sm), 128, 0, s>>>(
            (const int32_t *)rec.plans.ptr, (const int32_t *)rec.plan_steps.ptr, (const int64_t *)rec.op_off.ptr, ns,
            (int32_t *)rec.ops.ptr);
        PNE_CUDA_TRY(ctx, cudaGetLastError());
    }
    for (int64_t c = 0; c < n; ++c) rec.shape_count[shape[c]]++;
    // clusters by class, then shape (stable within a shape)
    const int n_cls = ok ? 1 + *std::max_element(shape_cls.begin(), shape_cls.end()) : 1;
    std::vector<int64_t> start(ns, 0);
    rec.class_start.assign(n_cls + 1, 0);
    rec.class_xmax.assign(n_cls, 0);
    {
        int64_t at = 0;
        for (int q = 0; q < n_cls; ++q) {
            rec.class_start[q] = at;
            rec.class_xmax[q] = kClassMin << q;
            for (int i = 0; i < ns; ++i)
                if (!ok || shape_cls[i] == q) { start[i] = at; at += rec.shape_count[i]; }
            if (!ok) break;
        }
        rec.class_start[n_cls] = at;
    }
    std::vector<int32_t> perm(n);
    for (int64_t c = 0; c < n; ++c) perm[start[shape[c]]++] = (int32_t)c;
    if ((st = dev_alloc(ctx, rec.perm, n * 4, s))) return st;
    if ((st = upload(ctx, rec.perm.ptr, perm.data(), n * 4, s))) return st;
    // per-cluster step tables
    if (ok) {
        int max_steps = 1;
        for (int i = 0; i < ns; ++i) max_steps = std::max(max_steps, stats[4 * i]);
        rec.step_stride = max_steps;
        dev_free(ctx, rec.step_off, s);
        dev_free(ctx, rec.step_site, s);
        if ((st = dev_alloc(ctx, rec.step_off, (size_t)n * max_steps * 4, s)) ||
            (st = dev_alloc(ctx, rec.step_site, (size_t)n * max_steps * 4, s)))
            return st;
        ContractParams cq = cp;
        cq.tens_off = g.d_tens_off; cq.blk_off = g.d_blk_off;
        cluster_steps_kernel<<<grid_for(n, 128, ctx->n_sm), 128, 0, s>>>(
            cq, (const int32_t *)sp.dshape.ptr, (const int32_t *)rec.plans.ptr, (const int32_t *)rec.plan_steps.ptr,
            max_steps, (int32_t *)rec.step_off.ptr, (int32_t *)rec.step_site.ptr);
        PNE_CUDA_TRY(ctx, cudaGetLastError());
    }
    rec.shape_of = sp.dshape;
    sp.dshape = DevBuf{};                 // the record owns it now
    rec.n_shapes = ns;
    rec.max_out = max_out;
    rec.shaped = ok && max_out <= 256;
    shapes_release(ctx, sp, s);
    return PNE_OK;
}

pne_status shapes_finish(pne_ctx *ctx, const Geometry &g, EnumRecord &rec, ShapePrep &sp, cudaStream_t s)
{
    pne_status st = shapes_plan(ctx, g, rec, sp, s);
    return st ? st : shapes_complete(ctx, g, rec, sp, s);
}

namespace {

// Multiply-adds of each cluster's plan (the algorithmic work of the contraction).
__global__ void __launch_bounds__(kCtWarps * 32) plan_work_kernel(ContractParams P, unsigned long long *total)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int *plan = (int *)smem_raw + wib * (kMaxSteps * kStepInts + kMaxSteps + 4);
    int *sites = plan + kMaxSteps * kStepInts;
    for (int64_t c = (int64_t)blockIdx.x * kCtWarps + wib; c < P.n_clusters; c += (int64_t)gridDim.x * kCtWarps) {
        if (lane == 0) {
            const int n = build_plan(P, c, plan, sites, kWarpTensorMax);
            unsigned long long f = 0;
            for (int t = 0; t < n; ++t) f += (unsigned long long)plan[t * kStepInts + 4] * plan[t * kStepInts + 5];
            atomicAdd(total, f);
        }
        __syncwarp();
    }
}

}  // namespace

pne_status launch_plan_work(pne_ctx *ctx, const pne_terms *t, cudaStream_t s, uint64_t *fma)
{
    const pne_partition *p = t->part;
    const EnumRecord &rec = *t->rec;
    *fma = 0;
    if (rec.n_clusters == 0) return PNE_OK;
    ContractParams cp;
    cp.n_clusters = (int64_t)rec.n_clusters; cp.n_members = 1; cp.n_sites = p->geo->closed.n_sites;
    cp.width = rec.width; cp.vwidth = rec.vwidth;
    cp.cl_edges = (const int32_t *)rec.cl_edges.ptr; cp.cl_verts = (const int32_t *)rec.cl_verts.ptr;
    cp.cl_size = (const int32_t *)rec.cl_size.ptr;
    cp.bond_site = p->geo->closed.d_bond_site; cp.bond_dim = p->geo->closed.d_bond_dim; cp.bond_leg = p->geo->closed.d_bond_leg;
    DevBuf tot;
    pne_status st = dev_alloc(ctx, tot, 8, s);
    if (st) return st;
    PNE_CUDA_TRY(ctx, cudaMemsetAsync(tot.ptr, 0, 8, s));
    const size_t smem = (size_t)kCtWarps * (kMaxSteps * kStepInts + kMaxSteps + 4) * 4;
    plan_work_kernel<<<grid_for(cp.n_clusters, kCtWarps, ctx->n_sm, 16), kCtWarps * 32, smem, s>>>(
        cp, (unsigned long long *)tot.ptr);
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    unsigned long long h = 0;
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(&h, tot.ptr, 8, cudaMemcpyDeviceToHost, s));
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    dev_free(ctx, tot, s);
    *fma = h;
    return PNE_OK;
}

namespace {

// Full-range blocks of the virtual geometry (bond dimensions d + 1) from the
// gauged blocked tensors: the block of leg set S holds T'_v / z_v with every
// leg outside S at 0 and every leg in S over its full range 0..d-1 (row-major,
// last leg fastest); each entry is the gauged entry of the same indices, which
// the blocked layout keeps in the block of its nonzero legs.  One warp per
// (member, site); index arithmetic only.
__global__ void comb_fill_kernel(const double *Mb, const int64_t *tens_off, const int32_t *blk_off, int64_t stride,
                                 const int64_t *vtens_off, const int32_t *vblk_off, int64_t vstride,
                                 const int32_t *site_ptr, const int32_t *site_bonds, const int32_t *bond_dim,
                                 int n_sites, int n_members, double *Mf)
{
    const int lane = threadIdx.x & 31;
    const int64_t items = (int64_t)n_members * n_sites;
    for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < items;
         item += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t member = item / n_sites;
        const int v = (int)(item % n_sites);
        const int l0 = site_ptr[v], k = site_ptr[v + 1] - l0;
        int d[kMaxDeg];
        for (int i = 0; i < k; ++i) d[i] = bond_dim[site_bonds[l0 + i]];
        const double *src = Mb + member * stride + tens_off[v];
        const int32_t *boff = blk_off + (int64_t)v * kBlkStride;
        const int32_t *vboff = vblk_off + (int64_t)v * kBlkStride;
        double *dst = Mf + member * vstride + vtens_off[v];
        for (int S = 0; S < (1 << k); ++S) {
            int n = 1;
            for (int i = 0; i < k; ++i) if (S >> i & 1) n *= d[i];
            for (int e = lane; e < n; e += 32) {
                int r = e, mask = 0, pos = 0, mul = 1;
                for (int i = k - 1; i >= 0; --i) {
                    if (!(S >> i & 1)) continue;
                    const int dgt = r % d[i];
                    r /= d[i];
                    if (dgt > 0) { mask |= 1 << i; pos += (dgt - 1) * mul; mul *= d[i] - 1; }
                }
                dst[vboff[S] + e] = src[boff[mask] + pos];
            }
        }
    }
}

}  // namespace

pne_status launch_contract(pne_ctx *ctx, pne_terms *t, int dtype, cudaStream_t s)
{
    const pne_partition *p = t->part;
    EnumRecord &rec = *t->rec;
    if (rec.n_clusters == 0) return PNE_OK;
    if (rec.comb) {
        // the combinatorial form: components contracted over the full range of
        // their bonds through the virtual geometry's blocks
        const Geometry &c = p->geo->closed, &vg = rec.vgeo;
        const int64_t vstride = vg.tens_off[vg.n_sites];
        const int64_t nf = (int64_t)p->n_members * vstride;
        pne_status st;
        if (!t->Mf.ptr && (st = dev_alloc(ctx, t->Mf, nf * 8, s))) return st;
        {
            ProfScope ps__(ctx, s, "comb_fill");
            const int64_t warps = (int64_t)p->n_members * c.n_sites;
            comb_fill_kernel<<<grid_for(warps * 32, 256, ctx->n_sm), 256, 0, s>>>(
                (const double *)p->Mb.ptr, c.d_tens_off, c.d_blk_off, c.tens_off[c.n_sites], vg.d_tens_off, vg.d_blk_off,
                vstride, c.d_site_ptr, c.d_site_bonds, c.d_bond_dim, c.n_sites, p->n_members, (double *)t->Mf.ptr);
        }
        PNE_LAUNCH_CHECK(ctx);
        const void *M = t->Mf.ptr;
        if (dtype == PNE_BF16) {
            if (!t->Mf16.ptr && (st = dev_alloc(ctx, t->Mf16, nf * 2, s))) return st;
            if ((st = convert_buffer(ctx, (const double *)t->Mf.ptr, nf, dtype, t->Mf16.ptr, s))) return st;
            M = t->Mf16.ptr;
        } else if (dtype != PNE_F64) {
            if (!t->Mf32.ptr && (st = dev_alloc(ctx, t->Mf32, nf * 4, s))) return st;
            if ((st = convert_buffer(ctx, (const double *)t->Mf.ptr, nf, dtype, t->Mf32.ptr, s))) return st;
            M = t->Mf32.ptr;
        }
        ContractParams cp;
        cp.n_clusters = (int64_t)rec.n_clusters; cp.n_members = p->n_members; cp.n_sites = c.n_sites;
        cp.width = rec.width; cp.vwidth = rec.vwidth;
        cp.cl_edges = (const int32_t *)rec.cl_edges.ptr; cp.cl_verts = (const int32_t *)rec.cl_verts.ptr;
        cp.cl_size = (const int32_t *)rec.cl_size.ptr;
        cp.bond_site = vg.d_bond_site; cp.bond_dim = vg.d_bond_dim; cp.bond_leg = vg.d_bond_leg;
        cp.blk_off = vg.d_blk_off; cp.tens_off = vg.d_tens_off; cp.stride = vstride;
        cp.scale = (const double *)p->site_scale.ptr; cp.zero = (const int8_t *)p->site_zero.ptr;
        cp.w = (double *)t->w.ptr; cp.nzc = (int32_t *)t->nzc.ptr; cp.status = (int32_t *)t->status.ptr;
        cp.M = M;
        ProfScope ps__(ctx, s, "contract");
        if (rec.shaped) {
            if (dtype == PNE_F64) return dispatch_shaped<double, Load<double>, 0>(ctx, cp, rec, s);
            if (dtype == PNE_BF16) return dispatch_shaped<float, LoadBF16, 2>(ctx, cp, rec, s);
            if (dtype == PNE_TF32) return dispatch_shaped<float, Load<float>, 1>(ctx, cp, rec, s);
            return dispatch_shaped<float, Load<float>, 0>(ctx, cp, rec, s);
        }
        if (dtype == PNE_F64) return run_general(ctx, contract_general_kernel<double, Load<double>, 0>, cp, 8, s);
        if (dtype == PNE_BF16) return run_general(ctx, contract_general_kernel<float, LoadBF16, 2>, cp, 4, s);
        if (dtype == PNE_TF32) return run_general(ctx, contract_general_kernel<float, Load<float>, 1>, cp, 4, s);
        return run_general(ctx, contract_general_kernel<float, Load<float>, 0>, cp, 4, s);
    }
    pne_status st = launch_convert(ctx, const_cast<pne_partition *>(p), dtype, s);
    if (st) return st;
    ContractParams cp;
    cp.n_clusters = (int64_t)rec.n_clusters; cp.n_members = p->n_members; cp.n_sites = p->geo->closed.n_sites;
    cp.width = rec.width; cp.vwidth = rec.vwidth;
    cp.cl_edges = (const int32_t *)rec.cl_edges.ptr; cp.cl_verts = (const int32_t *)rec.cl_verts.ptr;
    cp.cl_size = (const int32_t *)rec.cl_size.ptr;
    cp.bond_site = p->geo->closed.d_bond_site; cp.bond_dim = p->geo->closed.d_bond_dim; cp.bond_leg = p->geo->closed.d_bond_leg;
    cp.blk_off = p->geo->closed.d_blk_off; cp.tens_off = p->geo->closed.d_tens_off;
    cp.stride = p->geo->closed.tens_off[p->geo->closed.n_sites];
    cp.scale = (const double *)p->site_scale.ptr; cp.zero = (const int8_t *)p->site_zero.ptr;
    cp.w = (double *)t->w.ptr; cp.nzc = (int32_t *)t->nzc.ptr; cp.status = (int32_t *)t->status.ptr;
    const bool q1 = all_dims_two(p->geo->closed);
    ProfScope ps__(ctx, s, "contract");
    if (!q1 && rec.shaped) {
        if (dtype == PNE_F64) { cp.M = p->Mb.ptr; return dispatch_shaped<double, Load<double>, 0>(ctx, cp, rec, s); }
        if (dtype == PNE_BF16) { cp.M = p->Mb16.ptr; return dispatch_shaped<float, LoadBF16, 2>(ctx, cp, rec, s); }
        cp.M = p->Mb32.ptr;
        if (dtype == PNE_TF32) return dispatch_shaped<float, Load<float>, 1>(ctx, cp, rec, s);
        return dispatch_shaped<float, Load<float>, 0>(ctx, cp, rec, s);
    }
    if (dtype == PNE_F64) {
        cp.M = p->Mb.ptr;
        if (q1) contract_q1_kernel<double, Load<double>><<<grid_for(cp.n_clusters * cp.n_members, 256, ctx->n_sm), 256, 0, s>>>(cp);
        else return run_general(ctx, contract_general_kernel<double, Load<double>, 0>, cp, 8, s);
    } else if (dtype == PNE_BF16) {
        cp.M = p->Mb16.ptr;
        if (q1) contract_q1_kernel<float, LoadBF16><<<grid_for(cp.n_clusters * cp.n_members, 256, ctx->n_sm), 256, 0, s>>>(cp);
        else return run_general(ctx, contract_general_kernel<float, LoadBF16, 2>, cp, 4, s);
    } else {
        cp.M = p->Mb32.ptr;
        if (q1) contract_q1_kernel<float, Load<float>><<<grid_for(cp.n_clusters * cp.n_members, 256, ctx->n_sm), 256, 0, s>>>(cp);
        else if (dtype == PNE_TF32) return run_general(ctx, contract_general_kernel<float, Load<float>, 1>, cp, 4, s);
        else return run_general(ctx, contract_general_kernel<float, Load<float>, 0>, cp, 4, s);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}

// Small device regions gathered behind the sums' results, so that one
// device-to-host copy brings everything the host reads after the sums.
struct PackSegs {
    const char *src[4];
    int64_t off[4], bytes[4];
    int n;
};
__global__ void pack_segments_kernel(PackSegs P, char *dst)
{
    for (int q = 0; q < P.n; ++q)
        for (int64_t i = threadIdx.x; i < P.bytes[q]; i += blockDim.x) dst[P.off[q] + i] = P.src[q][i];
}

// per order k: the single clusters of size k, then every tuple level's terms
// of order k, in chunks of kSumChunk (the sum order of the per-order results)
std::vector<SumDesc> sum_descs(const EnumRecord &rec)
{
    std::vector<SumDesc> desc;
    const int K = rec.K;
    for (int k = 1; k <= K; ++k)
        for (int64_t b0 = rec.size_start[k]; b0 < rec.size_start[k + 1]; b0 += kSumChunk)
            desc.push_back({0, k, b0, std::min<int64_t>(b0 + kSumChunk, rec.size_start[k + 1])});
    for (size_t l = 0; l < rec.levels.size(); ++l)
        for (int k = 0; k <= K; ++k)
            for (int64_t b0 = rec.levels[l].order_start[k]; b0 < rec.levels[l].order_start[k + 1]; b0 += kSumChunk)
                desc.push_back({(int32_t)l + 1, k, b0, std::min<int64_t>(b0 + kSumChunk, rec.levels[l].order_start[k + 1])});
    return desc;
}

pne_status sum_desc_prepare(pne_ctx *ctx, EnumRecord &rec, cudaStream_t s)
{
    const std::vector<SumDesc> desc = sum_descs(rec);
    pne_status st;
    if (!desc.empty()) {
        if ((st = dev_alloc(ctx, rec.sum_desc, desc.size() * sizeof(SumDesc), s))) return st;
        if ((st = upload(ctx, rec.sum_desc.ptr, desc.data(), desc.size() * sizeof(SumDesc), s))) return st;
    }
    rec.n_sum_desc = (int)desc.size();
    return PNE_OK;
}

pne_status launch_sums(pne_ctx *ctx, const pne_terms *t, cudaStream_t s, std::vector<double> &c,
                       std::vector<double> &abs_c, int32_t *h_status, const std::vector<D2HCopy> &extra)
{
    const pne_partition *p = t->part;
    const int K = t->K, B = p->n_members;
    std::vector<SumDesc> desc;
    if (t->mode == PNE_MODE_ALL) {
        // handled by launch_all_mode; sums were written into t->sums
        std::vector<double> buf((size_t)B * (K + 1) * 2);
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(buf.data(), t->sums.ptr, buf.size() * 8, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h_status, t->status.ptr, 4, cudaMemcpyDeviceToHost, s));
        for (const D2HCopy &x : extra)
            PNE_CUDA_TRY(ctx, cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        c.assign((size_t)B * (K + 1), 0.0); abs_c.assign((size_t)B * (K + 1), 0.0);
        for (size_t i = 0; i < c.size(); ++i) { c[i] = buf[2 * i]; abs_c[i] = buf[2 * i + 1]; }
        return PNE_OK;
    }
    const EnumRecord &rec = *t->rec;
    if (rec.levels.size() > 16) { set_error(ctx, PNE_EOVERFLOW, "too many tuple levels"); return PNE_EOVERFLOW; }
    // the descriptors depend only on the record: built with it when it was
    // enumerated (already on the device), else here
    DevBuf dd, part, out;
    pne_status st;
    const SumDesc *d_desc = (const SumDesc *)rec.sum_desc.ptr;
    int nd = rec.n_sum_desc;
    if (nd < 0) {
        desc = sum_descs(rec);
        nd = (int)desc.size();
        if ((st = dev_alloc(ctx, dd, std::max(nd, 1) * sizeof(SumDesc), s))) return st;
        if (nd > 0 && (st = upload(ctx, dd.ptr, desc.data(), nd * sizeof(SumDesc), s))) return st;
        d_desc = (const SumDesc *)dd.ptr;
    }
    // out: the results [B][K+1][2], then the status word and the extra
    // regions, each at an 8-byte aligned offset
    const int64_t res_bytes = (int64_t)B * (K + 1) * 16;
    PackSegs segs{};
    int64_t tail = res_bytes;
    if (extra.size() > 3) { set_error(ctx, PNE_EINVAL, "too many read-back regions"); return PNE_EINVAL; }
    segs.src[0] = (const char *)t->status.ptr; segs.off[0] = tail; segs.bytes[0] = 4; tail += 8;
    segs.n = 1;
    for (const D2HCopy &x : extra) {
        segs.src[segs.n] = (const char *)x.src; segs.off[segs.n] = tail; segs.bytes[segs.n] = (int64_t)x.bytes;
        tail += ((int64_t)x.bytes + 7) & ~int64_t(7);
        ++segs.n;
    }
    if ((st = dev_alloc(ctx, part, (size_t)B * std::max(nd, 1) * 16, s))) return st;
    if ((st = dev_alloc(ctx, out, (size_t)tail, s))) return st;
    if (nd > 0 && !t->sum_done.ptr) {
        pne_terms *tm = const_cast<pne_terms *>(t);
        if ((st = dev_alloc(ctx, tm->sum_done, (size_t)B * 4, s))) return st;
        PNE_CUDA_TRY(ctx, cudaMemsetAsync(tm->sum_done.ptr, 0, (size_t)B * 4, s));
    }
    if (nd > 0) {
        SumParams sp;
        sp.desc = d_desc; sp.n_desc = nd; sp.n_members = B;
        sp.n_clusters = (int64_t)rec.n_clusters;
        sp.w = (const double *)t->w.ptr; sp.nzc = (const int32_t *)t->nzc.ptr;
        sp.vac = (const double *)p->vac.ptr;
        for (int l = 0; l < 16; ++l) { sp.lvl_idx[l] = nullptr; sp.lvl_m[l] = 0; }
        for (size_t l = 0; l < rec.levels.size(); ++l) {
            sp.lvl_idx[l] = (const int32_t *)rec.levels[l].idx.ptr;
            sp.lvl_m[l] = rec.levels[l].m;
        }
        sp.partial = (double *)part.ptr;
        sp.done = (unsigned int *)t->sum_done.ptr; sp.out = (double *)out.ptr; sp.K = K;
        if (B > 65535) { set_error(ctx, PNE_EINVAL, "too many tensor sets"); return PNE_EINVAL; }
        {
            ProfScope ps__(ctx, s, "term_sum");
            term_sum_kernel<<<dim3(nd, B), kSumThreads, 0, s>>>(sp);
        }
        PNE_CUDA_TRY(ctx, cudaGetLastError());
    } else {
        PNE_CUDA_TRY(ctx, cudaMemsetAsync(out.ptr, 0, (size_t)B * (K + 1) * 16, s));
    }
    pack_segments_kernel<<<1, 256, 0, s>>>(segs, (char *)out.ptr);
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    std::vector<double> buf((size_t)tail / 8);
    double *hb = (double *)pinned_slot(1, (size_t)tail);
    double *dst = hb ? hb : buf.data();
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(dst, out.ptr, (size_t)tail, cudaMemcpyDeviceToHost, s));
    dev_free(ctx, dd, s); dev_free(ctx, part, s); dev_free(ctx, out, s);
    {
        HostScope hw__(ctx, "sync_sum");
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    if (hb) std::memcpy(buf.data(), hb, (size_t)tail);
    const char *hbytes = (const char *)buf.data();
    std::memcpy(h_status, hbytes + segs.off[0], 4);
    for (size_t q = 0; q < extra.size(); ++q) std::memcpy(extra[q].dst, hbytes + segs.off[q + 1], extra[q].bytes);
    c.assign((size_t)B * (K + 1), 0.0); abs_c.assign((size_t)B * (K + 1), 0.0);
    for (size_t i = 0; i < c.size(); ++i) { c[i] = buf[2 * i]; abs_c[i] = buf[2 * i + 1]; }
    return PNE_OK;
}

pne_status launch_all_mode(pne_ctx *ctx, pne_terms *t, int dtype, cudaStream_t s)
{
    const pne_partition *p = t->part;
    const Geometry &g = p->geo->closed;
    const int K = t->K, B = p->n_members, Mc = g.n_bonds;
    if (Mc > kMaxAllBonds || g.n_sites > 64) {
        set_error(ctx, PNE_EINVAL, "ALL mode needs <= 30 closed bonds and <= 64 sites"); return PNE_EINVAL;
    }
    if (!all_dims_two(g)) {
        set_error(ctx, PNE_EINVAL, "ALL mode on the GPU needs bond dimension 2"); return PNE_EINVAL;
    }
    pne_status st = launch_convert(ctx, const_cast<pne_partition *>(p), dtype, s);
    if (st) return st;
    std::vector<int64_t> binom(31 * 31, 0);
    for (int n = 0; n <= 30; ++n) {
        binom[n * 31] = 1;
        for (int k = 1; k <= n; ++k) binom[n * 31 + k] = binom[(n - 1) * 31 + k - 1] + (k <= n - 1 ? binom[(n - 1) * 31 + k] : 0);
    }
    std::vector<SumDesc> desc;
    for (int k = 0; k <= std::min(K, Mc); ++k) {
        const int64_t nk = binom[Mc * 31 + k];
        for (int64_t b0 = 0; b0 < nk; b0 += kSumChunk) desc.push_back({0, k, b0, std::min<int64_t>(b0 + kSumChunk, nk)});
    }
    const int nd = (int)desc.size();
    DevBuf dd, bn, part, conn;
    if ((st = dev_alloc(ctx, dd, nd * sizeof(SumDesc), s))) return st;
    if ((st = dev_alloc(ctx, bn, binom.size() * 8, s))) return st;
    if ((st = dev_alloc(ctx, part, (size_t)B * nd * 16, s))) return st;
    if ((st = dev_alloc(ctx, conn, (size_t)nd * 8, s))) return st;
    if (!t->sums.ptr && (st = dev_alloc(ctx, t->sums, (size_t)B * (K + 1) * 16, s))) return st;
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(dd.ptr, desc.data(), nd * sizeof(SumDesc), cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bn.ptr, binom.data(), binom.size() * 8, cudaMemcpyHostToDevice, s));
    AllParams ap;
    ap.n_members = B; ap.n_sites = g.n_sites; ap.Mc = Mc; ap.K = K;
    ap.site_ptr = g.d_site_ptr; ap.site_bonds = g.d_site_bonds; ap.blk_off = g.d_blk_off;
    ap.tens_off = g.d_tens_off; ap.stride = g.tens_off[g.n_sites];
    ap.scale = (const double *)p->site_scale.ptr; ap.zero = (const int8_t *)p->site_zero.ptr;
    ap.vac = (const double *)p->vac.ptr; ap.binom = (const int64_t *)bn.ptr;
    ap.desc = (const SumDesc *)dd.ptr; ap.n_desc = nd; ap.partial = (double *)part.ptr;
    ap.conn_count = (int64_t *)conn.ptr; ap.bond_site = g.d_bond_site;
    {
        ProfScope ps_all__(ctx, s, "all_terms");
        if (dtype == PNE_F64) { ap.M = p->Mb.ptr; all_q1_kernel<double, Load<double>><<<dim3(nd, B), kSumThreads, 0, s>>>(ap); }
        else if (dtype == PNE_BF16) { ap.M = p->Mb16.ptr; all_q1_kernel<float, LoadBF16><<<dim3(nd, B), kSumThreads, 0, s>>>(ap); }
        else { ap.M = p->Mb32.ptr; all_q1_kernel<float, Load<float>><<<dim3(nd, B), kSumThreads, 0, s>>>(ap); }
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    {
        ProfScope ps__(ctx, s, "term_sum");
        finalize_kernel<<<grid_for((int64_t)B * (K + 1), 128, ctx->n_sm), 128, 0, s>>>(
        (const double *)part.ptr, (const SumDesc *)dd.ptr, nd, B, K, (double *)t->sums.ptr);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    std::vector<int64_t> hc(nd);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(hc.data(), conn.ptr, nd * 8, cudaMemcpyDeviceToHost, s));
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    uint64_t nconn = 0;
    for (int i = 0; i < nd; ++i) nconn += (uint64_t)hc[i];
    t->rec->n_clusters = nconn;
    dev_free(ctx, dd, s); dev_free(ctx, bn, s); dev_free(ctx, part, s); dev_free(ctx, conn, s);
    return PNE_OK;
}

}  // namespace pne


// ====================================================================== batched form
namespace pne {
namespace {

struct BatchGroup {
    ContractParams cp;
    int shaped;
    const int32_t *perm, *shape_of, *plans, *plan_steps, *ops, *step_off, *step_site;
    const int64_t *op_off;
    int step_stride;
    const double *vac;
    const int32_t *lvl_idx[8];
    int lvl_m[8];
    int K;
    int n_desc;
    int64_t desc_off, part_off, out_off;
};

struct BatchItem {
    int32_t g, kind, member, aux;   // kind 0: 32 clusters; kind 1: one sum descriptor (aux)
    int64_t start;
};

constexpr long long kBatchSpinLimit = 1ll << 26;

template <typename T, typename L, int R>
__device__ void lane_contract(const BatchGroup &G, int64_t i, int b, T *X0, T *X1)
{
    const ContractParams &P = G.cp;
    if (!G.shaped) {                                  // bond dimension 2: a plain product
        const int64_t c = i;
        const int32_t *E = P.cl_edges + c * P.width;
        const int32_t *V = P.cl_verts + c * P.vwidth;
        T prod = (T)1;
        int expo = 0, nz = 0;
        double zs = 1.0;
        for (int j = 0; j < P.vwidth && V[j] >= 0; ++j) {
            const int x = V[j];
            int mask = 0;
            for (int k = 0; k < P.width && E[k] >= 0; ++k) {
                const int e = E[k];
                if (P.bond_site[2 * e] == x) mask |= 1 << P.bond_leg[2 * e];
                if (P.bond_site[2 * e + 1] == x) mask |= 1 << P.bond_leg[2 * e + 1];
            }
            prod *= (T)L::get(P.M, (int64_t)b * P.stride + P.tens_off[x] + P.blk_off[x * kBlkStride + mask]);
            if (prod != (T)0) { int e; frexp((double)prod, &e); prod *= (T)pow2(-e); expo += e; }
            if (P.zero[(int64_t)b * P.n_sites + x]) { ++nz; zs *= P.scale[(int64_t)b * P.n_sites + x]; }
        }
        P.w[(int64_t)b * P.n_clusters + c] = ldexp((double)prod, expo) * zs;
        P.nzc[(int64_t)b * P.n_clusters + c] = nz;
        return;
    }
    const int64_t c = G.perm[i];
    const int sh = G.shape_of[c];
    shaped_cluster<T, L, R>(P, G.plans + (int64_t)sh * kPlanInts, G.plan_steps[sh], G.ops + G.op_off[sh],
                            G.step_off + c * G.step_stride, G.step_site + c * G.step_stride, c, b, X0, X1);
}

// The 32 clusters of a contraction item by groups of G lanes: 32 / G groups,
// group j taking clusters j, j + 32 / G, ... of the item; each group's
// running tensors sit in its slice of the warp's shared region W (2 * aux
// entries per group, within the 2 * 32 * xsm of the lane form).
template <typename T, typename L, int R, int G>
__device__ __forceinline__ void batch_groups(const BatchGroup &Gr, const BatchItem &wi, T *W, int lane)
{
    constexpr int NG = 32 / G;
    const int gi = lane / G, sub = lane % G;
    const unsigned gmask = group_mask<G>(lane);
    T *X = W + (int64_t)gi * 2 * wi.aux;
    T *Y = X + wi.aux;
    const ContractParams &P = Gr.cp;
    for (int k = 0; k < G; ++k) {
        const int64_t i = wi.start + gi + (int64_t)k * NG;
        if (i >= P.n_clusters) break;
        const int64_t c = Gr.perm[i];
        const int sh = Gr.shape_of[c];
        group_cluster<T, L, R, G>(P, Gr.plans + (int64_t)sh * kPlanInts, Gr.plan_steps[sh], Gr.ops + Gr.op_off[sh],
                                  Gr.step_off + c * Gr.step_stride, Gr.step_site + c * Gr.step_stride, c, wi.member,
                                  X, Y, sub, gmask);
    }
}

// One persistent launch: warps take items from one queue in order.  A sum item
// of handle g waits until every contraction item of g has been counted done;
// those items were taken earlier by running warps, so the wait ends.  It is
// bounded anyway: on timeout status[0] is set and the warp moves on.
template <typename T, typename L, int R>
__global__ void fused_batch_kernel(const BatchGroup *groups, const BatchItem *items, int64_t n_items,
                                   const SumDesc *descs, double *partials, unsigned long long *next,
                                   unsigned int *done, const unsigned int *need, int xsm, int xglob, T *xscratch,
                                   int32_t *status)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int wstride = max(8 * xsm, 16 * min(xsm, 16));         // shared entries per warp

    const int64_t gw = (int64_t)blockIdx.x * (blockDim.x >> 5) + wib;
    T *G0 = xscratch ? xscratch + gw * 2 * xglob * 32 + lane : nullptr;
    T *G1 = xscratch ? G0 + (int64_t)xglob * 32 : nullptr;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(next, 1ull);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= (unsigned long long)n_items) break;
        const BatchItem wi = items[it];
        const BatchGroup &G = groups[wi.g];
        if (wi.kind == 0) {
            const bool big = wi.aux > xsm;             // running tensors beyond the shared slices
            if (G.shaped && !big) {
                // groups of lanes per cluster in the warp's shared slices
                T *W = (T *)smem_raw + (int64_t)wib * wstride;
                if (wi.aux <= 16) batch_groups<T, L, R, 4>(G, wi, W, lane);
                else batch_groups<T, L, R, 8>(G, wi, W, lane);
            } else {
                // bond dimension 2 (no running tensor) or a running tensor in
                // the warp's global scratch
                const int64_t i = wi.start + lane;
                if (i < G.cp.n_clusters) lane_contract<T, L, R>(G, i, wi.member, G0, G1);
            }
            __syncwarp();
            if (lane == 0) { __threadfence(); atomicAdd(done + wi.g, 1u); }
        } else {
            if (lane == 0) {
                long long spins = 0;
                while (*((volatile unsigned int *)(done + wi.g)) < need[wi.g]) {
                    if (++spins > kBatchSpinLimit) { atomicExch(status + 1, 1); break; }
                    __nanosleep(100);
                }
                __threadfence();
            }
            __syncwarp();
            const SumDesc d = descs[G.desc_off + wi.aux];
            const int b = wi.member;
            const double *w = G.cp.w + (int64_t)b * G.cp.n_clusters;
            const int32_t *nzc = G.cp.nzc + (int64_t)b * G.cp.n_clusters;
            const int nzero = (int)G.vac[3 * b + 2];
            double sv = 0.0, av = 0.0;
            if (d.level == 0) {
                for (int64_t i = d.begin + lane; i < d.end; i += 32) {
                    const double v = (nzc[i] == nzero) ? w[i] : 0.0;
                    sv += v; av += fabs(v);
                }
            } else {
                const int m = G.lvl_m[d.level - 1];
                const int32_t *idx = G.lvl_idx[d.level - 1];
                for (int64_t i = d.begin + lane; i < d.end; i += 32) {
                    const int32_t *tp = idx + i * m;
                    double v = 1.0;
                    int z = 0;
                    for (int q = 0; q < m; ++q) { v *= w[tp[q]]; z += nzc[tp[q]]; }
                    if (z != nzero) v = 0.0;
                    sv += v; av += fabs(v);
                }
            }
            for (int off = 16; off > 0; off >>= 1) {
                sv += __shfl_xor_sync(0xffffffffu, sv, off);
                av += __shfl_xor_sync(0xffffffffu, av, off);
            }
            if (lane == 0) {
                double *p = partials + G.part_off + ((int64_t)b * G.n_desc + wi.aux) * 2;
                p[0] = sv; p[1] = av;
            }
        }
    }
}

__global__ void batch_finalize_kernel(const BatchGroup *groups, int G, const int64_t *fin_start,
                                      const SumDesc *descs, const double *partials, double *out)
{
    const int64_t total = fin_start[G];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = G;
        while (hi - lo > 1) { const int mid = (lo + hi) / 2; if (fin_start[mid] <= i) lo = mid; else hi = mid; }
        const BatchGroup &g = groups[lo];
        const int64_t r = i - fin_start[lo];
        const int b = (int)(r / (g.K + 1)), k = (int)(r % (g.K + 1));
        double sv = 0.0, av = 0.0;
        for (int d = 0; d < g.n_desc; ++d)
            if (descs[g.desc_off + d].order == k) {
                const double *p = partials + g.part_off + ((int64_t)b * g.n_desc + d) * 2;
                sv += p[0]; av += p[1];
            }
        double *o = out + g.out_off + (int64_t)b * ((g.K + 1) * 2 + 3);
        o[2 * k] = sv;
        o[2 * k + 1] = av;
        if (k == 0) { o[(g.K + 1) * 2] = g.vac[3 * b]; o[(g.K + 1) * 2 + 1] = g.vac[3 * b + 1]; o[(g.K + 1) * 2 + 2] = g.vac[3 * b + 2]; }
    }
}

}  // namespace

// counters block: next item (u64) | done[G] (u32) | need[G] (u32) | status[4] (i32, 16-aligned)
size_t status_offset(int G) { return ((size_t)8 + (size_t)8 * G + 15) & ~(size_t)15; }

// Running tensors of the fused batch live in shared memory up to kBatchSmemX
// entries, one pair per group of lanes (a warp's groups share one cluster
// item); items whose clusters need more use a per-warp slice of a global
// scratch buffer (one interleaved pair per lane), sized for the launch shape.
constexpr int kBatchSmemX = 32;

struct BatchPlan {
    int dtype = 0, G = 0, xmax = 1, xsm = 1;
    DevBuf xscratch;                    // [warps][2][xmax][32] elements, when xmax > xsm
    int64_t xscratch_warps = 0;
    int64_t n_items = 0, n_desc = 0, n_partials = 0, n_fin = 0, out_doubles = 0;
    std::vector<pne_terms *> terms;
    std::vector<int64_t> out_off;
    DevBuf groups, items, descs, partials, fin_start, counters, d_out;
    double *h_out = nullptr;
    size_t h_out_bytes = 0;
    size_t smem_per_warp = 0;
};

double *batch_host_out(BatchPlan *bp) { return bp->h_out; }
const std::vector<int64_t> &batch_out_offsets(BatchPlan *bp) { return bp->out_off; }

// The status words arrive with the results (read after the run's stream is
// synchronised): they sit right after the result doubles.
int32_t batch_status_host(BatchPlan *bp)
{
    const int32_t *st = (const int32_t *)(bp->h_out + std::max<int64_t>(bp->out_doubles, 1));
    return st[0] | st[1];
}

pne_status batch_plan_create(pne_ctx *ctx, const std::vector<pne_terms *> &terms, int dtype, cudaStream_t s,
                             BatchPlan **out)
{
    BatchPlan *bp = new BatchPlan();
    bp->dtype = dtype;
    bp->terms = terms;
    bp->G = (int)terms.size();
    std::vector<BatchGroup> groups(bp->G);
    std::vector<BatchItem> items;
    std::vector<SumDesc> descs;
    std::vector<int64_t> fin_start(bp->G + 1, 0);
    std::vector<unsigned int> need(bp->G, 0);
    std::vector<BatchItem> sum_items;
    int64_t part_off = 0, out_off = 0;
    pne_status st;
    for (int g = 0; g < bp->G; ++g) {
        pne_terms *t = terms[g];
        const pne_partition *p = t->part;
        const EnumRecord &rec = *t->rec;
        if (t->mode != PNE_MODE_LOOP) { delete bp; set_error(ctx, PNE_EINVAL, "batches take LOOP-mode handles"); return PNE_EINVAL; }
        const bool q1 = all_dims_two(p->geo->closed);
        if (!q1 && !rec.shaped && rec.n_clusters > 0) {
            delete bp; set_error(ctx, PNE_EINVAL, "a cluster exceeds the batched kernel's limits"); return PNE_EINVAL;
        }
        if ((st = launch_convert(ctx, const_cast<pne_partition *>(p), dtype, s))) { delete bp; return st; }
        BatchGroup &G = groups[g];
        ContractParams &cp = G.cp;
        cp.n_clusters = (int64_t)rec.n_clusters; cp.n_members = p->n_members; cp.n_sites = p->geo->closed.n_sites;
        cp.width = rec.width; cp.vwidth = rec.vwidth;
        cp.cl_edges = (const int32_t *)rec.cl_edges.ptr; cp.cl_verts = (const int32_t *)rec.cl_verts.ptr;
        cp.cl_size = (const int32_t *)rec.cl_size.ptr;
        cp.bond_site = p->geo->closed.d_bond_site; cp.bond_dim = p->geo->closed.d_bond_dim; cp.bond_leg = p->geo->closed.d_bond_leg;
        cp.blk_off = p->geo->closed.d_blk_off; cp.tens_off = p->geo->closed.d_tens_off; cp.stride = p->geo->closed.tens_off[p->geo->closed.n_sites];
        cp.M = dtype == PNE_F64 ? p->Mb.ptr : (dtype == PNE_BF16 ? p->Mb16.ptr : p->Mb32.ptr);
        cp.scale = (const double *)p->site_scale.ptr; cp.zero = (const int8_t *)p->site_zero.ptr;
        cp.w = (double *)t->w.ptr; cp.nzc = (int32_t *)t->nzc.ptr; cp.status = (int32_t *)t->status.ptr;
        G.shaped = (!q1 && rec.shaped) ? 1 : 0;
        G.perm = (const int32_t *)rec.perm.ptr; G.shape_of = (const int32_t *)rec.shape_of.ptr;
        G.plans = (const int32_t *)rec.plans.ptr; G.plan_steps = (const int32_t *)rec.plan_steps.ptr;
        G.ops = (const int32_t *)rec.ops.ptr; G.op_off = (const int64_t *)rec.op_off.ptr;
        G.step_off = (const int32_t *)rec.step_off.ptr; G.step_site = (const int32_t *)rec.step_site.ptr;
        G.step_stride = rec.step_stride;
        G.vac = (const double *)p->vac.ptr;
        for (int l = 0; l < 8; ++l) { G.lvl_idx[l] = nullptr; G.lvl_m[l] = 0; }
        if (rec.levels.size() > 8) { delete bp; set_error(ctx, PNE_EOVERFLOW, "too many tuple levels"); return PNE_EOVERFLOW; }
        for (size_t l = 0; l < rec.levels.size(); ++l) { G.lvl_idx[l] = (const int32_t *)rec.levels[l].idx.ptr; G.lvl_m[l] = rec.levels[l].m; }
        G.K = t->K;
        if (G.shaped) bp->xmax = std::max(bp->xmax, rec.max_out);
        // descriptors of this handle
        G.desc_off = (int64_t)descs.size();
        for (int k = 1; k <= t->K; ++k)
            for (int64_t b0 = rec.size_start[k]; b0 < rec.size_start[k + 1]; b0 += kSumChunk)
                descs.push_back({0, k, b0, std::min<int64_t>(b0 + kSumChunk, rec.size_start[k + 1])});
        for (size_t l = 0; l < rec.levels.size(); ++l)
            for (int k = 0; k <= t->K; ++k)
                for (int64_t b0 = rec.levels[l].order_start[k]; b0 < rec.levels[l].order_start[k + 1]; b0 += kSumChunk)
                    descs.push_back({(int32_t)l + 1, k, b0, std::min<int64_t>(b0 + kSumChunk, rec.levels[l].order_start[k + 1])});
        G.n_desc = (int)((int64_t)descs.size() - G.desc_off);
        G.part_off = part_off;
        part_off += (int64_t)p->n_members * G.n_desc * 2;
        G.out_off = out_off;
        bp->out_off.push_back(out_off);
        out_off += (int64_t)p->n_members * ((t->K + 1) * 2 + 3);
        fin_start[g + 1] = fin_start[g] + (int64_t)p->n_members * (t->K + 1);
        // items: contraction chunks of 32 clusters, then (later) the sums
        const int64_t chunks = (cp.n_clusters + 31) / 32;
        // running-tensor size an item needs: the class of its last cluster
        // (the clusters are listed by ascending class)
        std::vector<int32_t> chunk_x(chunks, 1);
        if (G.shaped)
            for (int64_t c = 0; c < chunks; ++c) {
                const int64_t last = std::min<int64_t>(c * 32 + 31, cp.n_clusters - 1);
                size_t q = 0;
                while (q + 2 < rec.class_start.size() && rec.class_start[q + 1] <= last) ++q;
                chunk_x[c] = std::min(rec.class_xmax[q], std::max(rec.max_out, 1));
            }
        for (int b = 0; b < p->n_members; ++b)
            for (int64_t c = 0; c < chunks; ++c) items.push_back({g, 0, b, chunk_x[c], c * 32});
        need[g] = (unsigned int)(chunks * p->n_members);
        for (int b = 0; b < p->n_members; ++b)
            for (int d = 0; d < G.n_desc; ++d) sum_items.push_back({g, 1, b, d, 0});
    }
    // the two work orders (PNE_SCHED_*), one after the other on the device:
    // handle order, then the contraction items by running-tensor size,
    // largest first (stable); the sum items follow the contraction items in both
    std::vector<BatchItem> largest(items);
    std::stable_sort(largest.begin(), largest.end(),
                     [](const BatchItem &a, const BatchItem &b) { return a.aux > b.aux; });
    items.insert(items.end(), sum_items.begin(), sum_items.end());
    largest.insert(largest.end(), sum_items.begin(), sum_items.end());
    bp->n_items = (int64_t)items.size();
    bp->n_desc = (int64_t)descs.size();
    bp->n_partials = part_off;
    bp->out_doubles = out_off;
    bp->n_fin = fin_start[bp->G];
    // counters: next (u64), done[G] (u32), need[G] (u32), status[2] (i32, 16-aligned)
    const size_t cnt_bytes = status_offset(bp->G) + 16;
    if ((st = dev_alloc(ctx, bp->groups, groups.size() * sizeof(BatchGroup), s)) ||
        (st = dev_alloc(ctx, bp->items, std::max<size_t>(2 * items.size(), 1) * sizeof(BatchItem), s)) ||
        (st = dev_alloc(ctx, bp->descs, std::max<size_t>(descs.size(), 1) * sizeof(SumDesc), s)) ||
        (st = dev_alloc(ctx, bp->partials, std::max<int64_t>(part_off, 1) * 8, s)) ||
        (st = dev_alloc(ctx, bp->fin_start, fin_start.size() * 8, s)) ||
        (st = dev_alloc(ctx, bp->counters, cnt_bytes, s)) ||
        (st = dev_alloc(ctx, bp->d_out, std::max<int64_t>(out_off, 1) * 8, s))) {
        batch_plan_destroy(ctx, bp, s);
        return st;
    }
    // results and the two status words, in pinned memory from the context's
    // pool (a cudaFreeHost per batch would synchronise the whole device)
    bp->h_out = (double *)take_pinned(ctx, (size_t)(std::max<int64_t>(out_off, 1) + 1) * 8, &bp->h_out_bytes);
    if (!bp->h_out) {
        batch_plan_destroy(ctx, bp, s);
        set_error(ctx, PNE_ENOMEM, "no pinned host memory for the batch results");
        return PNE_ENOMEM;
    }
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bp->groups.ptr, groups.data(), groups.size() * sizeof(BatchGroup), cudaMemcpyHostToDevice, s));
    if (!items.empty()) {
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bp->items.ptr, items.data(), items.size() * sizeof(BatchItem),
                                          cudaMemcpyHostToDevice, s));
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync((BatchItem *)bp->items.ptr + items.size(), largest.data(),
                                          largest.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, s));
    }
    if (!descs.empty()) PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bp->descs.ptr, descs.data(), descs.size() * sizeof(SumDesc), cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bp->fin_start.ptr, fin_start.data(), fin_start.size() * 8, cudaMemcpyHostToDevice, s));
    // need[] sits after next and done[]
    char *cb = (char *)bp->counters.ptr;
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(cb + 8 + (size_t)bp->G * 4, need.data(), (size_t)bp->G * 4, cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const size_t elem = (dtype == PNE_F64) ? 8 : 4;
    bp->xsm = std::min(bp->xmax, kBatchSmemX);
    // per warp: the running tensors of its lane groups (8 groups of 4 lanes,
    // 2 * aux entries each, for items up to 16 entries; 4 groups of 8 lanes for
    // items up to 32)
    bp->smem_per_warp = (size_t)std::max(8 * bp->xsm, 16 * std::min(bp->xsm, 16)) * elem;
    *out = bp;
    return PNE_OK;
}

namespace {
template <typename T, typename L, int R>
pne_status launch_fused(pne_ctx *ctx, BatchPlan *bp, int wpb, int bps, int sched, cudaStream_t s)
{
    auto kern = fused_batch_kernel<T, L, R>;
    const size_t smem = bp->smem_per_warp * wpb;
    grant_dynamic_smem((const void *)kern, smem);
    char *cb = (char *)bp->counters.ptr;
    unsigned long long *next = (unsigned long long *)cb;
    unsigned int *done = (unsigned int *)(cb + 8);
    const unsigned int *need = (const unsigned int *)(cb + 8 + (size_t)bp->G * 4);
    int32_t *status = (int32_t *)(cb + status_offset(bp->G));
    const bool glob = bp->xmax > bp->xsm;
    if (glob && bp->xscratch_warps < (int64_t)wpb * bps * ctx->n_sm) {
        set_error(ctx, PNE_EINVAL, "batch scratch not prepared for this launch shape");
        return PNE_EINVAL;
    }
    const BatchItem *items = (const BatchItem *)bp->items.ptr + (sched == PNE_SCHED_LARGEST_FIRST ? bp->n_items : 0);
    kern<<<bps * ctx->n_sm, wpb * 32, smem, s>>>((const BatchGroup *)bp->groups.ptr, items,
                                                 bp->n_items, (const SumDesc *)bp->descs.ptr, (double *)bp->partials.ptr,
                                                 next, done, need, bp->xsm, glob ? bp->xmax : 0,
                                                 glob ? (T *)bp->xscratch.ptr : nullptr, status);
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}
}  // namespace

int batch_max_blocks_per_sm(BatchPlan *bp, int wpb)
{
    int n = 0;
    const size_t smem = bp->smem_per_warp * wpb;
    if (smem > 200 * 1024) return 0;
    cudaError_t e;
    if (bp->dtype == PNE_F64) {
        grant_dynamic_smem((const void *)fused_batch_kernel<double, Load<double>, 0>, 200 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_batch_kernel<double, Load<double>, 0>, wpb * 32, smem);
    } else if (bp->dtype == PNE_BF16) {
        grant_dynamic_smem((const void *)fused_batch_kernel<float, LoadBF16, 2>, 200 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_batch_kernel<float, LoadBF16, 2>, wpb * 32, smem);
    } else {
        grant_dynamic_smem((const void *)fused_batch_kernel<float, Load<float>, 0>, 200 * 1024);
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fused_batch_kernel<float, Load<float>, 0>, wpb * 32, smem);
    }
    return e == cudaSuccess ? n : 0;
}

// The global running-tensor scratch for a launch shape (grow only; call
// before capturing a launch into a graph).
pne_status batch_prepare(pne_ctx *ctx, BatchPlan *bp, int wpb, int bps, cudaStream_t s)
{
    if (bp->xmax <= bp->xsm) return PNE_OK;
    const int64_t warps = (int64_t)wpb * bps * ctx->n_sm;
    if (warps <= bp->xscratch_warps) return PNE_OK;
    const size_t elem = (bp->dtype == PNE_F64) ? 8 : 4;
    dev_free(ctx, bp->xscratch, s);
    bp->xscratch_warps = 0;
    pne_status st = dev_alloc(ctx, bp->xscratch, (size_t)warps * 2 * bp->xmax * 32 * elem, s);
    if (st) return st;
    bp->xscratch_warps = warps;
    return PNE_OK;
}

pne_status batch_enqueue(pne_ctx *ctx, BatchPlan *bp, int wpb, int bps, int sched, cudaStream_t s)
{
    pne_status st;
    // conversions of updated partitions (each partition once)
    std::vector<const pne_partition *> seen;
    for (pne_terms *t : bp->terms) {
        if (std::find(seen.begin(), seen.end(), t->part) != seen.end()) continue;
        seen.push_back(t->part);
        if ((st = launch_convert_only(ctx, t->part, bp->dtype, s))) return st;
    }
    char *cb = (char *)bp->counters.ptr;
    PNE_CUDA_TRY(ctx, cudaMemsetAsync(cb, 0, 8 + (size_t)bp->G * 4, s));
    PNE_CUDA_TRY(ctx, cudaMemsetAsync(cb + status_offset(bp->G), 0, 16, s));
    {
        ProfScope ps(ctx, s, "batch_fused");
        if (bp->dtype == PNE_F64) st = launch_fused<double, Load<double>, 0>(ctx, bp, wpb, bps, sched, s);
        else if (bp->dtype == PNE_BF16) st = launch_fused<float, LoadBF16, 2>(ctx, bp, wpb, bps, sched, s);
        else if (bp->dtype == PNE_TF32) st = launch_fused<float, Load<float>, 1>(ctx, bp, wpb, bps, sched, s);
        else st = launch_fused<float, Load<float>, 0>(ctx, bp, wpb, bps, sched, s);
        if (st) return st;
    }
    {
        ProfScope ps(ctx, s, "batch_finalize");
        batch_finalize_kernel<<<grid_for(bp->n_fin, 128, ctx->n_sm), 128, 0, s>>>(
            (const BatchGroup *)bp->groups.ptr, bp->G, (const int64_t *)bp->fin_start.ptr, (const SumDesc *)bp->descs.ptr,
            (const double *)bp->partials.ptr, (double *)bp->d_out.ptr);
        PNE_CUDA_TRY(ctx, cudaGetLastError());
    }
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bp->h_out, bp->d_out.ptr, std::max<int64_t>(bp->out_doubles, 1) * 8,
                                      cudaMemcpyDeviceToHost, s));
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(bp->h_out + std::max<int64_t>(bp->out_doubles, 1),
                                      (char *)bp->counters.ptr + status_offset(bp->G), 8, cudaMemcpyDeviceToHost, s));
    return PNE_OK;
}

void batch_plan_destroy(pne_ctx *ctx, BatchPlan *bp, cudaStream_t s)
{
    if (!bp) return;
    DevBuf *bufs[] = {&bp->groups, &bp->items, &bp->descs, &bp->partials, &bp->fin_start, &bp->counters, &bp->d_out,
                      &bp->xscratch};
    for (DevBuf *b : bufs) dev_free(ctx, *b, s);
    if (bp->h_out) {
        // the last copy into the pinned result buffer may still be queued
        cudaStreamSynchronize(s);
        give_pinned(ctx, bp->h_out, bp->h_out_bytes);
    }
    delete bp;
}

}  // namespace pne
