// Bond partitions on the GPU: belief propagation, the symmetrising gauge and
// the excitation-blocked layout of the gauged site tensors.  All FP64.
//
// * BP (Sec. I, Sec. II.B): Jacobi sweeps; each outgoing message of a site is
//   its tensor contracted with the messages arriving on its other legs,
//   normalised to unit 2-norm with the largest-magnitude entry positive.  An
//   open index reflects the site's own outgoing message back (Sec. III.D).
//   One persistent cooperative launch runs every sweep of every tensor set,
//   with a bounded grid barrier between sweeps.
// * Gauge (App. B): for bond b = (s0, s1) with outgoing messages m0 (of s0)
//   and m1 (of s1), n = <m0|m1>.  x = [m0^T / n ; R_perp] where R_perp holds
//   d-1 orthonormal rows orthogonal to m1 (rows 1.. of the Householder
//   reflector that maps m1 to a multiple of e0).  Then x m1 = e0 and
//   e0^T x = m0^T / n, so in the new basis P_b = e0 e0^T (Eq. A7) and
//   Q_b = diag(0, 1, .., 1).  x^{-1} has the closed form
//   [m1 | R_perp^T - m1 (R_perp m0)^T / n].
//   s0's leg is multiplied by x^{-1}, s1's leg by x^T (from the left).
// * Blocked layout: entries of a gauged site tensor are grouped by the set S
//   of legs whose index is >= 1 ("excited"); block S is the dense sub-tensor
//   over those legs with index values 1..d-1.  A cluster contraction reads
//   exactly one block per site.  Each site is divided by z_v (its all-zero
//   entry) when z_v != 0, else by a power of two.
#include <cuda_runtime.h>
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include <atomic>

#include "pne_internal.h"

namespace pne {

namespace {

constexpr int kBpWarps = 8;              // warps per block in the BP kernels
// warps per block of the cluster form: 4 with two sites per warp task, 8 with one
template <int TASK> struct ClusterForm {
    static constexpr int kWarps = TASK == 2 ? 4 : 8;
    // resident blocks per SM the register budget allows: 96 registers for the
    // pair form (a few spilled) leave room on every SM for the enumeration's
    // kernels that run beside the sweeps; at 128 the step was 1% slower
    static constexpr int kMinBlocks = TASK == 2 ? 5 : 4;
};
// shared memory per block up to which the cluster form keeps its warps' site
// tensors resident (four blocks per SM still fit in 228 KB)
constexpr size_t kBpTensorSmem = 48 * 1024;
constexpr long long kBarrierSpinLimit = 1ll << 25;

struct BPParams {
    int n_sets, n_sites, n_legs;
    const int32_t *site_ptr, *site_bonds, *bond_dim, *inc_slot;
    const int64_t *tens_off;
    int64_t set_stride;
    const double *T;
    double *msg;                  // [2][n_sets][n_legs][8]
    double tol, damping;
    int max_iter;
    unsigned long long *res;      // [4][n_sets] residual of sweep it in slot it % 4
    int32_t *done_it;             // [n_sets] iteration of convergence (0: not yet)
    int32_t *iters_out;           // [n_sets]
    double *res_out;              // [n_sets]
    int32_t *final_buf;           // [n_sets]
    int32_t *flags;               // [0] barrier timeout, [1] degenerate message
    unsigned int *bar;            // [0] count, [1] generation
    int n_colors;                 // > 0: colour-ordered sweeps, in place; 0: Jacobi, two buffers
    const int32_t *color_ptr, *color_sites;
    int smem_per_warp;            // doubles
    int tabA, tabC;               // table sizes (max over sites)
};

// Grid-wide barrier for a cooperative launch.  The wait is bounded: on timeout
// flags[0] is set and every block leaves its loop at the next check.
__device__ bool grid_barrier(unsigned int *bar, int32_t *flags, unsigned int nblocks)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *gen = bar + 1;
        unsigned int g = *gen;
        __threadfence();
        unsigned int arrived = atomicAdd(bar, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g) {
                if (++spins > kBarrierSpinLimit) { atomicExch(flags, 1); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *((volatile int32_t *)flags) == 0;
}

// All outgoing messages of one site, warp-cooperative.
// The legs are split in two halves H1 = [0,h), H2 = [h,k).  X1 = T contracted
// with the incoming messages on H2 (a tensor over H1), X2 = T contracted on H1
// (over H2).  An output on a leg of H1 is X1 contracted with the messages on
// the other legs of H1, and likewise for H2.
__device__ void site_messages(const double *__restrict__ T, int k, const int *dims,
                              const double *in, double *u, double *w, double *x1, double *x2,
                              double *out, int lane)
{
    int h = k / 2;
    int A = 1, C = 1;
    for (int i = 0; i < h; ++i) A *= dims[i];
    for (int i = h; i < k; ++i) C *= dims[i];
    // outer-product weight tables
    float inv[kMaxDeg];
    for (int i = 0; i < k; ++i) inv[i] = 1.0f / (float)dims[i];
    for (int c = lane; c < C; c += 32) {
        int r = c, m;
        double p = 1.0;
        for (int i = k - 1; i >= h; --i) { r = fdivmod(r, dims[i], inv[i], m); p *= in[i * kMsgStride + m]; }
        w[c] = p;
    }
    for (int a = lane; a < A; a += 32) {
        int r = a, m;
        double p = 1.0;
        for (int i = h - 1; i >= 0; --i) { r = fdivmod(r, dims[i], inv[i], m); p *= in[i * kMsgStride + m]; }
        u[a] = p;
    }
    __syncwarp();
    // X1[a] = sum_c T[a][c] w[c]: lpr lanes share a row (consecutive lanes),
    // each summing a strided part of it, then a fixed shuffle tree
    {
        int lpr = 1;
        while (lpr * 2 * A <= 32) lpr *= 2;
        const int rows_per_pass = 32 / lpr, sub = lane % lpr;
        for (int a0 = 0; a0 < A; a0 += rows_per_pass) {
            const int a = a0 + lane / lpr;
            double s = 0.0;
            if (a < A) {
                const double *row = T + (int64_t)a * C;
                for (int c = sub; c < C; c += lpr) s = fma(row[c], w[c], s);
            }
            for (int off = lpr / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (a < A && sub == 0) x1[a] = s;
        }
    }
    // X2[c] = sum_a u[a] T[a][c]: lpc lanes share a column, split over a
    {
        int lpc = 1;
        while (lpc * 2 * C <= 32) lpc *= 2;
        const int cols_per_pass = 32 / lpc;
        const int sub = lane / cols_per_pass;           // lanes of one column are cols_per_pass apart
        for (int c0 = 0; c0 < C; c0 += cols_per_pass) {
            const int c = c0 + lane % cols_per_pass;
            double s = 0.0;
            if (c < C)
                for (int a = sub; a < A; a += lpc) s = fma(u[a], T[(int64_t)a * C + c], s);
            for (int off = 16; off >= cols_per_pass; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (c < C && sub == 0) x2[c] = s;
        }
    }
    __syncwarp();
    // outputs: one (leg, value) pair per lane
    int n_items = 0;
    for (int j = 0; j < k; ++j) n_items += dims[j];
    for (int it = lane; it < n_items; it += 32) {
        int j = 0, x = it;
        while (x >= dims[j]) { x -= dims[j]; ++j; }
        const double *X = (j < h) ? x1 : x2;
        int lo = (j < h) ? 0 : h, hi = (j < h) ? h : k;
        int size = (j < h) ? A : C;
        int stride = 1;
        for (int i = hi - 1; i > j; --i) stride *= dims[i];
        int rest = size / dims[j];
        const float inv_stride = 1.0f / (float)stride;
        double s = 0.0;
        for (int r = 0; r < rest; ++r) {
            int rs;
            const int qs = fdivmod(r, stride, inv_stride, rs);
            int a = qs * (stride * dims[j]) + x * stride + rs;
            double p = X[a];
            int rr = a, dgt;
            for (int i = hi - 1; i >= lo; --i) {
                rr = fdivmod(rr, dims[i], inv[i], dgt);
                if (i != j) p *= in[i * kMsgStride + dgt];
            }
            s += p;
        }
        out[j * kMsgStride + x] = s;
    }
    __syncwarp();
}

__global__ void bp_init_kernel(double *msg, const int32_t *site_ptr, const int32_t *site_bonds,
                               const int32_t *bond_dim, int n_sites, int n_legs, int n_sets)
{
    int64_t total = (int64_t)n_sets * n_legs;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        int slot = (int)(i % n_legs);
        int d = bond_dim[site_bonds[slot]];
        double v = 1.0 / sqrt((double)d);
        for (int a = 0; a < kMsgStride; ++a) msg[i * kMsgStride + a] = (a < d) ? v : 0.0;
    }
}

__global__ void __launch_bounds__(kBpWarps * 32) bp_persistent_kernel(BPParams p)
{
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *ws = smem + wib * p.smem_per_warp;
    double *in = ws;                       // [6][8]
    double *out = in + kMaxDeg * kMsgStride;  // [6][8]
    double *u = out + kMaxDeg * kMsgStride;
    double *w = u + p.tabA;
    double *x1 = w + p.tabC;
    double *x2 = x1 + p.tabA;
    const unsigned int nblocks = gridDim.x;
    const int64_t gwarp = (int64_t)blockIdx.x * kBpWarps + wib;
    const int64_t nwarps = (int64_t)nblocks * kBpWarps;
    const int64_t msg_set = (int64_t)p.n_legs * kMsgStride;
    const int64_t msg_buf = (int64_t)p.n_sets * msg_set;
    const bool colored = p.n_colors > 0;
    const int phases = colored ? p.n_colors : 1;

    for (int it = 1; it <= p.max_iter; ++it) {
        const int src = colored ? 0 : (it - 1) & 1, dst = colored ? 0 : it & 1;
        // Slots it%4 (this sweep) and (it-1)%4 are live here; a slower block may
        // still read (it-2)%4 in its bookkeeping of the previous sweep.  Slot
        // (it+1)%4 was last read before the previous barrier: clear it now.
        unsigned long long *res_cur = p.res + (int64_t)(it % 4) * p.n_sets;
        unsigned long long *res_prev = p.res + (int64_t)((it + 3) % 4) * p.n_sets;
        if (blockIdx.x == 0) {
            unsigned long long *res_next = p.res + (int64_t)((it + 1) % 4) * p.n_sets;
            for (int s = threadIdx.x; s < p.n_sets; s += blockDim.x) res_next[s] = 0ull;
        }
        for (int ph = 0; ph < phases; ++ph) {
        const int c0 = colored ? p.color_ptr[ph] : 0;
        const int nc = colored ? p.color_ptr[ph + 1] - c0 : p.n_sites;
        const int64_t items = (int64_t)p.n_sets * nc;
        for (int64_t item = gwarp; item < items; item += nwarps) {
            const int set = (int)(item / nc), q = (int)(item % nc);
            const int v = colored ? p.color_sites[c0 + q] : q;
            if (p.done_it[set] != 0) continue;
            if (it > 1 && __longlong_as_double((long long)res_prev[set]) < p.tol) continue;
            const int l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
            int dims[kMaxDeg];
            for (int i = 0; i < kMaxDeg; ++i) dims[i] = (i < k) ? p.bond_dim[p.site_bonds[l0 + i]] : 1;
            const double *msrc = p.msg + src * msg_buf + set * msg_set;
            double *mdst = p.msg + dst * msg_buf + set * msg_set;
            for (int e = lane; e < k * kMsgStride; e += 32) {
                int i = e / kMsgStride, a = e % kMsgStride;
                in[e] = msrc[(int64_t)p.inc_slot[l0 + i] * kMsgStride + a];
            }
            __syncwarp();
            const double *T = p.T + set * p.set_stride + p.tens_off[v];
            site_messages(T, k, dims, in, u, w, x1, x2, out, lane);
            // normalise every message in parallel: lane = (leg j, entry a), 8 lanes per leg
            double r = 0.0;
            for (int j0 = 0; j0 < k; j0 += 4) {
                const int j = j0 + (lane >> 3), a = lane & 7;
                const bool live = (j < k) && (a < dims[j < k ? j : 0]);
                const double o = live ? out[j * kMsgStride + a] : 0.0;
                const double old = live ? msrc[(int64_t)(l0 + j) * kMsgStride + a] : 0.0;
                double n2 = o * o;
                for (int off = 4; off > 0; off >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, off);
                // sign: the entry of largest magnitude, first index on ties
                double big = live ? fabs(o) : -1.0;
                int arg = a;
                for (int off = 4; off > 0; off >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, big, off);
                    const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
                    if (ob > big || (ob == big && oa < arg)) { big = ob; arg = oa; }
                }
                const double oarg = __shfl_sync(0xffffffffu, o, (lane & ~7) | arg);
                double nrm = sqrt(n2);
                if (j < k && !(nrm > 0.0)) { atomicExch(p.flags + 1, 1); nrm = 1.0; }
                double nv = (oarg < 0.0 ? -o : o) / nrm;
                if (p.damping > 0.0) {
                    double m = (1.0 - p.damping) * nv + p.damping * old;
                    double m2 = live ? m * m : 0.0;
                    for (int off = 4; off > 0; off >>= 1) m2 += __shfl_xor_sync(0xffffffffu, m2, off);
                    double bg = live ? fabs(m) : -1.0;
                    int ag = a;
                    for (int off = 4; off > 0; off >>= 1) {
                        const double ob = __shfl_xor_sync(0xffffffffu, bg, off);
                        const int oa = __shfl_xor_sync(0xffffffffu, ag, off);
                        if (ob > bg || (ob == bg && oa < ag)) { bg = ob; ag = oa; }
                    }
                    const double marg = __shfl_sync(0xffffffffu, m, (lane & ~7) | ag);
                    double n3 = sqrt(m2);
                    if (j < k && !(n3 > 0.0)) { atomicExch(p.flags + 1, 1); n3 = 1.0; }
                    nv = (marg < 0.0 ? -m : m) / n3;
                }
                if (live) {
                    mdst[(int64_t)(l0 + j) * kMsgStride + a] = nv;
                    r = fmax(r, fabs(nv - old));
                }
            }
            for (int off = 16; off > 0; off >>= 1) r = fmax(r, __shfl_xor_sync(0xffffffffu, r, off));
            if (lane == 0) atomicMax(res_cur + set, (unsigned long long)__double_as_longlong(r));
            __syncwarp();
        }
        if (ph + 1 < phases && !grid_barrier(p.bar, p.flags, nblocks)) return;
        }
        if (!grid_barrier(p.bar, p.flags, nblocks)) return;
        // convergence bookkeeping: every warp reads the residuals one set per
        // lane and reaches the same decision; warp 0 of block 0 records
        bool all_done = true;
        const bool recorder = blockIdx.x == 0 && threadIdx.x < 32;
        for (int s0 = 0; s0 < p.n_sets; s0 += 32) {
            const int s = s0 + (threadIdx.x & 31);
            bool pending = false;
            if (s < p.n_sets) {
                const bool was = p.done_it[s] != 0 ||
                                 (it > 1 && __longlong_as_double((long long)res_prev[s]) < p.tol);
                if (!was) {
                    const double rs = __longlong_as_double((long long)res_cur[s]);
                    if (rs < p.tol) {
                        if (recorder) { p.done_it[s] = it; p.iters_out[s] = it; p.res_out[s] = rs; p.final_buf[s] = dst; }
                    } else {
                        pending = true;
                        if (it == p.max_iter && recorder) { p.iters_out[s] = 0; p.res_out[s] = rs; p.final_buf[s] = dst; }
                    }
                }
            }
            if (__any_sync(0xffffffffu, pending)) all_done = false;
        }
        if (all_done) return;
    }
}

// ---------------------------------------------------------------- float-float sweeps
// The same Jacobi sweeps with every multiply and add carried as an unevaluated
// sum of two FP32 numbers (hi + lo): products by Dekker's error-free product
// (one FMA recovers the rounding error of a*b), sums by Knuth's error-free
// two-sum, dot products accumulated with a compensation term.  About 2^-48
// relative precision per operation, on the FP32 pipes (64x the FP64 rate of
// this part).  Site tensors are pre-scaled by a power of two per site (the
// normalised messages do not change); messages live as (hi, lo) pairs.
struct ff { float h, l; };

__device__ __forceinline__ ff ff_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ ff ff_fast(float a, float b)        // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ ff ff_mul(ff x, ff y)
{
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fadd_rn(e, __fmaf_rn(x.h, y.l, __fmul_rn(x.l, y.h)));
    return ff_fast(p, e);
}
__device__ __forceinline__ ff ff_add(ff x, ff y)
{
    const ff s = ff_two_sum(x.h, y.h), t = ff_two_sum(x.l, y.l);
    const ff v = ff_fast(s.h, __fadd_rn(s.l, t.h));
    return ff_fast(v.h, __fadd_rn(t.l, v.l));
}
// compensated accumulator: value = h + c
struct ffacc {
    float h = 0.f, c = 0.f;
    __device__ __forceinline__ void add(ff p)
    {
        const ff s = ff_two_sum(h, p.h);
        h = s.h;
        c = __fadd_rn(c, __fadd_rn(s.l, p.l));
    }
    __device__ __forceinline__ ff get() const { return ff_fast(h, c); }
    // += x y: the exact product's low part goes to the compensation term
    // without being renormalised first (12 FP32 instructions)
    __device__ __forceinline__ void mad(ff x, ff y)
    {
        const float q = __fmul_rn(x.h, y.h);
        float e = __fmaf_rn(x.h, y.h, -q);
        e = __fmaf_rn(x.h, y.l, __fmaf_rn(x.l, y.h, e));
        const ff s = ff_two_sum(h, q);
        h = s.h;
        c = __fadd_rn(c, __fadd_rn(s.l, e));
    }
};
__device__ __forceinline__ ff ff_shfl_xor(ff x, int off)
{
    return {__shfl_xor_sync(0xffffffffu, x.h, off), __shfl_xor_sync(0xffffffffu, x.l, off)};
}
__device__ __forceinline__ ff ff_sqrt(ff x)
{
    if (!(x.h > 0.f)) return {0.f, 0.f};
    const float s = sqrtf(x.h);
    const float r = __fadd_rn(__fmaf_rn(-s, s, x.h), x.l);
    return ff_fast(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}
__device__ __forceinline__ ff ff_div(ff x, ff y)
{
    const float q1 = __fdiv_rn(x.h, y.h);
    const ff r = ff_add(x, ff_mul({-q1, 0.f}, y));
    return ff_fast(q1, __fdiv_rn(r.h, y.h));
}
// |x| > |y| (lexicographic on the normalised pair)
__device__ __forceinline__ bool ff_abs_gt(ff x, ff y)
{
    if (x.h < 0.f) { x.h = -x.h; x.l = -x.l; }
    if (y.h < 0.f) { y.h = -y.h; y.l = -y.l; }
    return x.h > y.h || (x.h == y.h && x.l > y.l);
}

// x * 2^-ex as a float-float pair (hi = x rounded to nearest-even in FP32, lo =
// the remainder rounded), from the bits of x with integer operations only: no
// FP64 instruction.  Requires |x| * 2^-ex <= 1 (ex at least the slice's
// largest exponent).  Parts below FP32's normal range are flushed to zero:
// entries 2^-126 below the slice maximum (hi) or 2^-74 below it (lo) carry
// nothing the pair precision could keep anyway.
__device__ __forceinline__ ff split_scaled(double x, int ex)
{
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FF);
    const int e2 = E - 1023 - ex;                       // exponent of the scaled value
    if (E == 0 || e2 < -126) return {0.f, 0.f};
    const unsigned long long m = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    unsigned long long q = m >> 29;                     // top 24 bits
    const unsigned long long r = m & ((1ull << 29) - 1);
    if (r > (1ull << 28) || (r == (1ull << 28) && (q & 1))) ++q;
    const int rem = (int)((long long)m - (long long)(q << 29));   // |rem| <= 2^28
    int eh = e2;
    if (q == (1ull << 24)) { q >>= 1; ++eh; }
    const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
    const float hi = __int_as_float((int)(sign | ((unsigned)(eh + 127) << 23) | (unsigned)(q & 0x7FFFFF)));
    float lo = 0.f;
    if (rem != 0 && e2 - 52 >= -126) {
        lo = __fmul_rn(__int2float_rn(rem), __int_as_float((e2 - 52 + 127) << 23));
        if (sign) lo = -lo;
    }
    return {hi, lo};
}

// a normal FP32 value widened to FP64 from its bits (zero stays zero)
__device__ __forceinline__ double widen(float f)
{
    const unsigned u = (unsigned)__float_as_int(f);
    const unsigned e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    const unsigned long long bits = ((unsigned long long)(u >> 31) << 63) |
                                    ((unsigned long long)(e + 1023 - 127) << 52) |
                                    ((unsigned long long)(u & 0x7FFFFF) << 29);
    return __longlong_as_double((long long)bits);
}

struct BPFFParams {
    int n_sets, n_sites, n_legs;
    const int32_t *site_ptr, *site_bonds, *bond_dim, *inc_slot;
    const int64_t *tens_off;
    int64_t set_stride;
    const ff *T;                  // [n_sets][stride] scaled, float-float
    ff *msg;                      // [2][n_sets][n_legs][8]
    float tol;
    double damping;
    int max_iter;
    unsigned int *res;            // [4][n_sets] float bits
    int32_t *done_it, *iters_out, *final_buf, *flags;
    double *res_out;
    unsigned int *bar;
    int n_colors;                 // as in BPParams
    const int32_t *color_ptr, *color_sites;
    int smem_per_warp;            // ff entries
    int tabA, tabC;
    // cluster form: each warp's site tensors kept in shared memory across the
    // sweeps (t_slots per warp of slot_ff entries, slot_ff even); 0 = read
    // them from global memory every sweep
    int t_slots, slot_ff;
    double *msg64;                // cluster form: the final messages in FP64, buffer 0 ([n_sets][n_legs][8])
};

__device__ void site_messages_ff(const ff *__restrict__ T, int k, const int *dims, const ff *in, ff *u, ff *w,
                                 ff *x1, ff *x2, ff *out, int lane)
{
    const int h = k / 2;
    int A = 1, C = 1;
    for (int i = 0; i < h; ++i) A *= dims[i];
    for (int i = h; i < k; ++i) C *= dims[i];
    float inv[kMaxDeg];
    for (int i = 0; i < k; ++i) inv[i] = 1.0f / (float)dims[i];
    for (int c = lane; c < C; c += 32) {
        int r = c, m;
        ff p = {1.f, 0.f};
        for (int i = k - 1; i >= h; --i) { r = fdivmod(r, dims[i], inv[i], m); p = ff_mul(p, in[i * kMsgStride + m]); }
        w[c] = p;
    }
    for (int a = lane; a < A; a += 32) {
        int r = a, m;
        ff p = {1.f, 0.f};
        for (int i = h - 1; i >= 0; --i) { r = fdivmod(r, dims[i], inv[i], m); p = ff_mul(p, in[i * kMsgStride + m]); }
        u[a] = p;
    }
    __syncwarp();
    {
        int lpr = 1;
        while (lpr * 2 * A <= 32) lpr *= 2;
        const int rows_per_pass = 32 / lpr, sub = lane % lpr;
        for (int a0 = 0; a0 < A; a0 += rows_per_pass) {
            const int a = a0 + lane / lpr;
            ffacc acc;
            if (a < A) {
                const ff *row = T + (int64_t)a * C;
                for (int c = sub; c < C; c += lpr) acc.mad(row[c], w[c]);
            }
            ff s = acc.get();
            for (int off = lpr / 2; off > 0; off >>= 1) s = ff_add(s, ff_shfl_xor(s, off));
            if (a < A && sub == 0) x1[a] = s;
        }
    }
    {
        int lpc = 1;
        while (lpc * 2 * C <= 32) lpc *= 2;
        const int cols_per_pass = 32 / lpc, sub = lane / cols_per_pass;
        for (int c0 = 0; c0 < C; c0 += cols_per_pass) {
            const int c = c0 + lane % cols_per_pass;
            ffacc acc;
            if (c < C)
                for (int a = sub; a < A; a += lpc) acc.mad(u[a], T[(int64_t)a * C + c]);
            ff s = acc.get();
            for (int off = 16; off >= cols_per_pass; off >>= 1) s = ff_add(s, ff_shfl_xor(s, off));
            if (c < C && sub == 0) x2[c] = s;
        }
    }
    __syncwarp();
    int n_items = 0;
    for (int j = 0; j < k; ++j) n_items += dims[j];
    for (int it = lane; it < n_items; it += 32) {
        int j = 0, x = it;
        while (x >= dims[j]) { x -= dims[j]; ++j; }
        const ff *X = (j < h) ? x1 : x2;
        const int lo = (j < h) ? 0 : h, hi = (j < h) ? h : k, size = (j < h) ? A : C;
        int stride = 1;
        for (int i = hi - 1; i > j; --i) stride *= dims[i];
        const int rest = size / dims[j];
        const float inv_stride = 1.0f / (float)stride;
        ffacc acc;
        for (int r = 0; r < rest; ++r) {
            int rs;
            const int qs = fdivmod(r, stride, inv_stride, rs);
            const int a = qs * (stride * dims[j]) + x * stride + rs;
            ff p = X[a];
            int rr = a, dgt;
            for (int i = hi - 1; i >= lo; --i) {
                rr = fdivmod(rr, dims[i], inv[i], dgt);
                if (i != j) p = ff_mul(p, in[i * kMsgStride + dgt]);
            }
            acc.add(p);
        }
        out[j * kMsgStride + x] = acc.get();
    }
    __syncwarp();
}

// ---- the same site update with the leg count K and a uniform bond dimension D
// known at compile time (the lattice sites: every index decode is a constant
// division, every loop bound a constant).  Same halves, same outputs.
__host__ __device__ constexpr int cpow(int b, int e) { return e == 0 ? 1 : b * cpow(b, e - 1); }
__host__ __device__ constexpr int lanes_for(int rows) { return rows >= 32 ? 1 : (rows > 16 ? 1 : (rows > 8 ? 2 : (rows > 4 ? 4 : (rows > 2 ? 8 : (rows > 1 ? 16 : 32))))); }

// out for leg jj of a half with NL legs: sum over the other digits of X times
// the messages on the other legs of the half (inh: the half's first message row)
template <int NL, int D>
__device__ __forceinline__ ff half_output(const ff *X, const ff *inh, int jj, int x)
{
    constexpr int REST = cpow(D, NL - 1);
    ffacc acc;
#pragma unroll 4
    for (int r = 0; r < REST; ++r) {
        // digits of the legs other than jj, last leg fastest; leg jj takes x
        int rr = r, a = 0, mul = 1;
        ff p = {1.f, 0.f};
        bool first = true;
#pragma unroll
        for (int i = NL - 1; i >= 0; --i) {
            int dgt;
            if (i == jj) {
                dgt = x;
            } else {
                dgt = rr % D;
                rr /= D;
                const ff m = inh[i * kMsgStride + dgt];
                p = first ? m : ff_mul(p, m);
                first = false;
            }
            a += dgt * mul;
            mul *= D;
        }
        acc.add(first ? X[a] : ff_mul(X[a], p));
    }
    return acc.get();
}

template <int K, int D>
__device__ void site_messages_ff_u(const ff *__restrict__ T, const ff *in, ff *u, ff *w, ff *x1, ff *x2, ff *out,
                                   int lane)
{
    constexpr int H = K / 2, A = cpow(D, H), C = cpow(D, K - H);
    for (int c = lane; c < C; c += 32) {
        int r = c;
        ff q = {1.f, 0.f};
#pragma unroll
        for (int i = K - 1; i >= H; --i) { q = ff_mul(q, in[i * kMsgStride + r % D]); r /= D; }
        w[c] = q;
    }
    for (int a = lane; a < A; a += 32) {
        int r = a;
        ff q = {1.f, 0.f};
#pragma unroll
        for (int i = H - 1; i >= 0; --i) { q = ff_mul(q, in[i * kMsgStride + r % D]); r /= D; }
        u[a] = q;
    }
    __syncwarp();
    {   // x1 = T w: LPR lanes per row
        constexpr int LPR = lanes_for(A), RPP = 32 / LPR;
        const int sub = lane % LPR;
#pragma unroll 1
        for (int a0 = 0; a0 < A; a0 += RPP) {
            const int a = a0 + lane / LPR;
            ffacc acc;
            if (a < A) {
                const ff *row = T + (int64_t)a * C;
#pragma unroll 4
                for (int c = sub; c < C; c += LPR) acc.mad(row[c], w[c]);
            }
            ff sm = acc.get();
#pragma unroll
            for (int off = LPR / 2; off > 0; off >>= 1) sm = ff_add(sm, ff_shfl_xor(sm, off));
            if (a < A && sub == 0) x1[a] = sm;
        }
    }
    {   // x2 = u^T T: LPC lanes per column
        constexpr int LPC = lanes_for(C), CPP = 32 / LPC;
        const int sub = lane / CPP;
#pragma unroll 1
        for (int c0 = 0; c0 < C; c0 += CPP) {
            const int c = c0 + lane % CPP;
            ffacc acc;
            if (c < C) {
#pragma unroll 4
                for (int a = sub; a < A; a += LPC) acc.mad(u[a], T[(int64_t)a * C + c]);
            }
            ff sm = acc.get();
#pragma unroll
            for (int off = 16; off >= CPP; off >>= 1) sm = ff_add(sm, ff_shfl_xor(sm, off));
            if (c < C && sub == 0) x2[c] = sm;
        }
    }
    __syncwarp();
    for (int it = lane; it < K * D; it += 32) {
        const int j = it / D, x = it % D;
        out[j * kMsgStride + x] = (j < H) ? half_output<H, D>(x1, in, j, x)
                                          : half_output<K - H, D>(x2, in + H * kMsgStride, j - H, x);
    }
    __syncwarp();
}

// the specialised update when the site's legs share one dimension of a
// compiled (K, D) pair; false otherwise (the caller takes the general routine)
__device__ __forceinline__ bool site_messages_ff_fast(const ff *T, int k, const int *dims, const ff *in, ff *u, ff *w,
                                                      ff *x1, ff *x2, ff *out, int lane)
{
    const int D = dims[0];
    for (int i = 1; i < k; ++i)
        if (dims[i] != D) return false;
    switch (k * 16 + D) {
#define PNE_SITE_CASE(KK, DD) case KK * 16 + DD: site_messages_ff_u<KK, DD>(T, in, u, w, x1, x2, out, lane); return true;
        PNE_SITE_CASE(2, 2) PNE_SITE_CASE(2, 3) PNE_SITE_CASE(2, 4) PNE_SITE_CASE(2, 5) PNE_SITE_CASE(2, 6)
        PNE_SITE_CASE(3, 2) PNE_SITE_CASE(3, 3) PNE_SITE_CASE(3, 4) PNE_SITE_CASE(3, 5) PNE_SITE_CASE(3, 6)
        PNE_SITE_CASE(4, 2) PNE_SITE_CASE(4, 3) PNE_SITE_CASE(4, 4) PNE_SITE_CASE(4, 5) PNE_SITE_CASE(4, 6)
        PNE_SITE_CASE(5, 2) PNE_SITE_CASE(5, 3) PNE_SITE_CASE(5, 4)
        PNE_SITE_CASE(6, 2) PNE_SITE_CASE(6, 3) PNE_SITE_CASE(6, 4)
#undef PNE_SITE_CASE
        default: return false;
    }
}

__device__ __forceinline__ ff ldcg_ff(const ff *q)
{
    const float2 v = __ldcg(reinterpret_cast<const float2 *>(q));
    return {v.x, v.y};
}

// Normalisation of a site's outgoing messages, LPL lanes per leg (LPL = 4
// when every leg has dimension <= 4, else 8): unit 2-norm, the largest |entry|
// positive (first index on ties), optional damping against the old message,
// written to mdst; returns the largest entry change (the same in every lane).
template <int LPL>
__device__ __forceinline__ float ff_normalise_write(const BPFFParams &p, int l0, int k, const int *dims, const ff *msrc,
                                                    ff *mdst, const ff *out, int lane)
{
    constexpr int LPW = 32 / LPL;
    float r = 0.f;
    for (int j0 = 0; j0 < k; j0 += LPW) {
        const int j = j0 + lane / LPL, a = lane % LPL;
        const bool live = (j < k) && (a < dims[j < k ? j : 0]);
        const ff o = live ? out[j * kMsgStride + a] : ff{0.f, 0.f};
        const ff old = live ? ldcg_ff(&msrc[(int64_t)(l0 + j) * kMsgStride + a]) : ff{0.f, 0.f};
        ff n2 = ff_mul(o, o);
#pragma unroll
        for (int off = LPL / 2; off > 0; off >>= 1) n2 = ff_add(n2, ff_shfl_xor(n2, off));
        ff big = live ? o : ff{-1.f, 0.f};
        bool has = live;
        int arg = a;
#pragma unroll
        for (int off = LPL / 2; off > 0; off >>= 1) {
            const ff ob = ff_shfl_xor(big, off);
            const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
            const bool oh = __shfl_xor_sync(0xffffffffu, has, off);
            const bool take = oh && (!has || ff_abs_gt(ob, big) || (!ff_abs_gt(big, ob) && oa < arg));
            if (take) { big = ob; arg = oa; has = true; }
        }
        const float oarg = __shfl_sync(0xffffffffu, o.h, (lane & ~(LPL - 1)) | arg);
        ff nrm = ff_sqrt(n2);
        if (j < k && !(nrm.h > 0.f)) { atomicExch(p.flags + 1, 1); nrm = {1.f, 0.f}; }
        ff nv = ff_div(oarg < 0.f ? ff{-o.h, -o.l} : o, nrm);
        if (p.damping > 0.0) {
            const float dm = (float)p.damping;
            ff m = ff_add(ff_mul(nv, {1.f - dm, 0.f}), ff_mul(old, {dm, 0.f}));
            ff m2 = live ? ff_mul(m, m) : ff{0.f, 0.f};
#pragma unroll
            for (int off = LPL / 2; off > 0; off >>= 1) m2 = ff_add(m2, ff_shfl_xor(m2, off));
            ff bg = live ? m : ff{-1.f, 0.f};
            bool hs = live;
            int ag = a;
#pragma unroll
            for (int off = LPL / 2; off > 0; off >>= 1) {
                const ff ob = ff_shfl_xor(bg, off);
                const int oa = __shfl_xor_sync(0xffffffffu, ag, off);
                const bool oh = __shfl_xor_sync(0xffffffffu, hs, off);
                const bool take = oh && (!hs || ff_abs_gt(ob, bg) || (!ff_abs_gt(bg, ob) && oa < ag));
                if (take) { bg = ob; ag = oa; hs = true; }
            }
            const float marg = __shfl_sync(0xffffffffu, m.h, (lane & ~(LPL - 1)) | ag);
            ff n3 = ff_sqrt(m2);
            if (j < k && !(n3.h > 0.f)) { atomicExch(p.flags + 1, 1); n3 = {1.f, 0.f}; }
            nv = ff_div(marg < 0.f ? ff{-m.h, -m.l} : m, n3);
        }
        if (live) {
            mdst[(int64_t)(l0 + j) * kMsgStride + a] = nv;
            r = fmaxf(r, fabsf(__fadd_rn(__fsub_rn(nv.h, old.h), __fsub_rn(nv.l, old.l))));
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
    return r;
}

// ---- sites whose legs all have dimension 4 (2 to 4 legs), two per warp.
// Half h = lane >> 4 of the warp updates its own site; inside a half, lane
// hl = 4 rg + cg holds rows rg RA .. rg RA + RA - 1 and columns cg RC ..
// cg RC + RC - 1 of T[a][c] (a over the first H = K / 2 legs, c over the
// others, last leg fastest), so each entry is read once for both halves of the
// contraction: x1 = T w over the lane's columns and x2 = u^T T over its rows,
// then summed over the four lanes of a row group (x1) or of a column group
// (x2).  The same lane hl then forms output entry x = cg of leg j = rg and
// normalises it with the other three lanes of its leg.  A site's result does
// not depend on the other half's site (or on whether there is one).

// the four values v[0..3] summed over the lanes that differ in lane bits hi
// and lo; lane keeps the sum of v[2 bit(hi) + bit(lo)]
__device__ __forceinline__ ff ff_reduce_scatter4(ff v0, ff v1, ff v2, ff v3, int lane, int hi, int lo)
{
    const bool bh = (lane & hi) != 0, bl = (lane & lo) != 0;
    const ff k0 = ff_add(bh ? v2 : v0, ff_shfl_xor(bh ? v0 : v2, hi));
    const ff k1 = ff_add(bh ? v3 : v1, ff_shfl_xor(bh ? v1 : v3, hi));
    return ff_add(bl ? k1 : k0, ff_shfl_xor(bl ? k0 : k1, lo));
}
// v summed over the lanes that differ in lane bits hi and lo (the same in all four)
__device__ __forceinline__ ff ff_allreduce4(ff v, int hi, int lo)
{
    v = ff_add(v, ff_shfl_xor(v, hi));
    return ff_add(v, ff_shfl_xor(v, lo));
}

// largest |entry| of the four lanes of a leg (first index on ties), as in
// ff_normalise_write; returns the lane offset (0..3) of that entry
__device__ __forceinline__ int ff_argmax4(ff v, bool live, int a)
{
    ff big = live ? v : ff{-1.f, 0.f};
    bool has = live;
    int arg = a;
#pragma unroll
    for (int off = 2; off > 0; off >>= 1) {
        const ff ob = ff_shfl_xor(big, off);
        const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
        const bool oh = __shfl_xor_sync(0xffffffffu, has, off);
        const bool take = oh && (!has || ff_abs_gt(ob, big) || (!ff_abs_gt(big, ob) && oa < arg));
        if (take) { big = ob; arg = oa; has = true; }
    }
    return arg;
}

// Per-slot records of the cluster form, in shared memory: kSlotMeta ints
// (first leg, pair kind, site id, the legs' incoming message slots) and the
// site's current outgoing messages [4][4] (the entries this warp last wrote).
constexpr int kSlotMeta = 8;
enum { kMetaL0 = 0, kMetaKind = 1, kMetaSite = 2, kMetaInc = 3 };

// RC consecutive pair entries from 16-byte aligned (RC = 4) or 8-byte aligned
// (RC = 1) shared memory
template <int RC> __device__ __forceinline__ void ff_load_row(const ff *row, ff *t);
template <> __device__ __forceinline__ void ff_load_row<4>(const ff *row, ff *t)
{
    const float4 a = reinterpret_cast<const float4 *>(row)[0], b = reinterpret_cast<const float4 *>(row)[1];
    t[0] = {a.x, a.y}; t[1] = {a.z, a.w}; t[2] = {b.x, b.y}; t[3] = {b.z, b.w};
}
template <> __device__ __forceinline__ void ff_load_row<1>(const ff *row, ff *t)
{
    const float2 a = *reinterpret_cast<const float2 *>(row);
    t[0] = {a.x, a.y};
}

// every lane passes its half's site (meta, cur: the slot's records; T: its
// tensor, 16-byte aligned; live: false for a half with no site of its own,
// which then repeats the other half's site without writing); ws: the warp's
// scratch, >= 128 ff.  Returns the largest message change over both sites
// (the same in every lane).
template <int K>
__device__ float ff_site_pair4(const BPFFParams &p, const int *meta, ff *cur, const ff *__restrict__ T, bool live,
                               ff *msg, ff *ws, int lane)
{
    constexpr int H = K / 2, A = cpow(4, H), C = cpow(4, K - H), RA = A / 4, RC = C / 4;
    const int h = lane >> 4, hl = lane & 15, rg = hl >> 2, cg = hl & 3;
    ff *in = ws + h * 32;             // [K][kMsgStride]
    ff *x1 = ws + 64 + h * 16;        // [A]
    ff *x2 = ws + 96 + h * 16;        // [C]
    const int j = rg, x = cg;         // the lane's output entry
    const bool mine = live && j < K;
    const int l0 = meta[kMetaL0];
    ff old = {0.f, 0.f};
    if (j < K) {
        in[j * kMsgStride + x] = ldcg_ff(&msg[(int64_t)meta[kMetaInc + j] * kMsgStride + x]);
        old = cur[j * 4 + x];
    }
    __syncwarp();
    ff w[RC];
    if constexpr (K - H == 2) {
        const ff b = in[H * kMsgStride + cg];
#pragma unroll
        for (int i = 0; i < 4; ++i) w[i] = ff_mul(b, in[(H + 1) * kMsgStride + i]);
    } else {
        w[0] = in[H * kMsgStride + cg];
    }
    ffacc p1[RA], p2[RC];
#pragma unroll
    for (int r = 0; r < RA; ++r) {
        const ff ur = (H == 2) ? ff_mul(in[rg], in[kMsgStride + r]) : in[rg];
        const ff *row = T + (rg * RA + r) * C + cg * RC;
        ff t[RC];
        ff_load_row<RC>(row, t);
#pragma unroll
        for (int i = 0; i < RC; ++i) {
            p1[r].mad(t[i], w[i]);
            p2[i].mad(ur, t[i]);
        }
    }
    if constexpr (RA == 4) {
        x1[4 * rg + cg] = ff_reduce_scatter4(p1[0].get(), p1[1].get(), p1[2].get(), p1[3].get(), lane, 2, 1);
    } else {
        const ff s1 = ff_allreduce4(p1[0].get(), 2, 1);
        if (cg == 0) x1[rg] = s1;
    }
    if constexpr (RC == 4) {
        x2[4 * cg + rg] = ff_reduce_scatter4(p2[0].get(), p2[1].get(), p2[2].get(), p2[3].get(), lane, 8, 4);
    } else {
        const ff s2 = ff_allreduce4(p2[0].get(), 8, 4);
        if (rg == 0) x2[cg] = s2;
    }
    __syncwarp();
    // output entry x of leg j: a one-leg half is x1 / x2 itself; in a two-leg
    // half, the sum over the half's other leg times its message
    ff o = {0.f, 0.f};
    if (j < K) {
        const bool first = j < H;
        const ff *X = first ? x1 : x2;
        if ((first ? H : K - H) == 1) {
            o = X[x];
        } else {
            const int jj = first ? j : j - H;
            const ff *m = in + (first ? 1 - j : H + 1 - jj) * kMsgStride;
            ffacc acc;
#pragma unroll
            for (int y = 0; y < 4; ++y) acc.mad(X[jj ? 4 * y + x : 4 * x + y], m[y]);
            o = acc.get();
        }
    }
    // unit 2-norm over the leg's four lanes, largest |entry| positive
    ff n2 = ff_mul(o, o);
    n2 = ff_allreduce4(n2, 2, 1);
    const int arg = ff_argmax4(o, j < K, x);
    const float oarg = __shfl_sync(0xffffffffu, o.h, (lane & ~3) | arg);
    ff nrm = ff_sqrt(n2);
    if (mine && !(nrm.h > 0.f)) atomicExch(p.flags + 1, 1);
    if (!(nrm.h > 0.f)) nrm = {1.f, 0.f};
    ff nv = ff_div(oarg < 0.f ? ff{-o.h, -o.l} : o, nrm);
    if (p.damping > 0.0) {
        const float dm = (float)p.damping;
        const ff m = ff_add(ff_mul(nv, {1.f - dm, 0.f}), ff_mul(old, {dm, 0.f}));
        ff m2 = ff_allreduce4(ff_mul(m, m), 2, 1);
        const int ag = ff_argmax4(m, j < K, x);
        const float marg = __shfl_sync(0xffffffffu, m.h, (lane & ~3) | ag);
        ff n3 = ff_sqrt(m2);
        if (mine && !(n3.h > 0.f)) atomicExch(p.flags + 1, 1);
        if (!(n3.h > 0.f)) n3 = {1.f, 0.f};
        nv = ff_div(marg < 0.f ? ff{-m.h, -m.l} : m, n3);
    }
    float r = 0.f;
    __syncwarp();
    if (mine) {
        msg[(int64_t)(l0 + j) * kMsgStride + x] = nv;
        cur[j * 4 + x] = nv;
        r = fabsf(__fadd_rn(__fsub_rn(nv.h, old.h), __fsub_rn(nv.l, old.l)));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
    return r;
}

// 2, 3 or 4 when every leg of v has dimension 4 (the pair form above), else 0
__device__ __forceinline__ int ff_pair_kind(const BPFFParams &p, int v)
{
    const int l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
    if (k < 2 || k > 4) return 0;
    for (int i = 0; i < k; ++i)
        if (p.bond_dim[p.site_bonds[l0 + i]] != 4) return 0;
    return k;
}

__device__ __forceinline__ float ff_pair_dispatch(const BPFFParams &p, int kind, const int *meta, ff *cur, const ff *T,
                                                  bool live, ff *msg, ff *ws, int lane)
{
    switch (kind) {
        case 2: return ff_site_pair4<2>(p, meta, cur, T, live, msg, ws, lane);
        case 3: return ff_site_pair4<3>(p, meta, cur, T, live, msg, ws, lane);
        default: return ff_site_pair4<4>(p, meta, cur, T, live, msg, ws, lane);
    }
}

// One site's outgoing messages, normalised and written to mdst; returns the
// largest entry change (the same in every lane).  Messages are read through L2
// (__ldcg): other blocks wrote them earlier in the same launch.  Tv is the
// site's tensor (in global or shared memory).
__device__ float ff_site_update(const BPFFParams &p, int v, const ff *Tv, const ff *msrc, ff *mdst, ff *in, ff *out,
                                ff *u, ff *w, ff *x1, ff *x2, int lane)
{
    const int l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
    int dims[kMaxDeg];
    int dmax = 1;
    for (int i = 0; i < kMaxDeg; ++i) {
        dims[i] = (i < k) ? p.bond_dim[p.site_bonds[l0 + i]] : 1;
        dmax = dims[i] > dmax ? dims[i] : dmax;
    }
    for (int e = lane; e < k * kMsgStride; e += 32)
        in[e] = ldcg_ff(&msrc[(int64_t)p.inc_slot[l0 + e / kMsgStride] * kMsgStride + e % kMsgStride]);
    __syncwarp();
    if (!site_messages_ff_fast(Tv, k, dims, in, u, w, x1, x2, out, lane))
        site_messages_ff(Tv, k, dims, in, u, w, x1, x2, out, lane);
    return dmax <= 4 ? ff_normalise_write<4>(p, l0, k, dims, msrc, mdst, out, lane)
                     : ff_normalise_write<8>(p, l0, k, dims, msrc, mdst, out, lane);
}

__global__ void __launch_bounds__(kBpWarps * 32, 4) bp_ff_kernel(BPFFParams p)
{
    extern __shared__ __align__(16) ff ffsmem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    ff *ws = ffsmem + wib * p.smem_per_warp;
    ff *in = ws;
    ff *out = in + kMaxDeg * kMsgStride;
    ff *u = out + kMaxDeg * kMsgStride;
    ff *w = u + p.tabA;
    ff *x1 = w + p.tabC;
    ff *x2 = x1 + p.tabA;
    const unsigned int nblocks = gridDim.x;
    const int64_t gwarp = (int64_t)blockIdx.x * kBpWarps + wib, nwarps = (int64_t)nblocks * kBpWarps;
    const int64_t msg_set = (int64_t)p.n_legs * kMsgStride, msg_buf = (int64_t)p.n_sets * msg_set;
    const bool colored = p.n_colors > 0;
    const int phases = colored ? p.n_colors : 1;
    for (int it = 1; it <= p.max_iter; ++it) {
        const int src = colored ? 0 : (it - 1) & 1, dst = colored ? 0 : it & 1;
        unsigned int *res_cur = p.res + (int64_t)(it % 4) * p.n_sets;
        unsigned int *res_prev = p.res + (int64_t)((it + 3) % 4) * p.n_sets;
        if (blockIdx.x == 0) {
            unsigned int *res_next = p.res + (int64_t)((it + 1) % 4) * p.n_sets;
            for (int s = threadIdx.x; s < p.n_sets; s += blockDim.x) res_next[s] = 0u;
        }
        for (int ph = 0; ph < phases; ++ph) {
        const int c0 = colored ? p.color_ptr[ph] : 0;
        const int nc = colored ? p.color_ptr[ph + 1] - c0 : p.n_sites;
        const int64_t items = (int64_t)p.n_sets * nc;
        for (int64_t item = gwarp; item < items; item += nwarps) {
            const int set = (int)(item / nc), q = (int)(item % nc);
            const int v = colored ? p.color_sites[c0 + q] : q;
            if (__ldcg(p.done_it + set) != 0) continue;
            if (it > 1 && __uint_as_float(__ldcg(res_prev + set)) < p.tol) continue;
            const ff *msrc = p.msg + src * msg_buf + set * msg_set;
            ff *mdst = p.msg + dst * msg_buf + set * msg_set;
            const float r = ff_site_update(p, v, p.T + set * p.set_stride + p.tens_off[v], msrc, mdst, in, out, u,
                                           w, x1, x2, lane);
            if (lane == 0) atomicMax(res_cur + set, __float_as_uint(r));
            __syncwarp();
        }
        if (ph + 1 < phases && !grid_barrier(p.bar, p.flags, nblocks)) return;
        }
        if (!grid_barrier(p.bar, p.flags, nblocks)) return;
        // convergence bookkeeping, one set per lane (as in the FP64 kernel)
        bool all_done = true;
        const bool recorder = blockIdx.x == 0 && threadIdx.x < 32;
        for (int s0 = 0; s0 < p.n_sets; s0 += 32) {
            const int s = s0 + lane;
            bool pending = false;
            if (s < p.n_sets) {
                const bool was = __ldcg(p.done_it + s) != 0 || (it > 1 && __uint_as_float(__ldcg(res_prev + s)) < p.tol);
                if (!was) {
                    const float rs = __uint_as_float(__ldcg(res_cur + s));
                    if (rs < p.tol) {
                        if (recorder) { p.done_it[s] = it; p.iters_out[s] = it; p.res_out[s] = (double)rs; p.final_buf[s] = dst; }
                    } else {
                        pending = true;
                        if (it == p.max_iter && recorder) { p.iters_out[s] = 0; p.res_out[s] = (double)rs; p.final_buf[s] = dst; }
                    }
                }
            }
            if (__any_sync(0xffffffffu, pending)) all_done = false;
        }
        if (all_done) return;
    }
}

// Float-float BP with one thread-block cluster per tensor set: the cluster's
// warps share the set's sites of one colour, and the hardware cluster barrier
// separates the colour phases, so no grid-wide barrier is needed and every set
// stops at its own convergence (the other sets do not wait for it).  Colour
// order only (in place, buffer 0).  Every block of a cluster takes the same
// path: the loop decision depends only on the set's residual, read after a
// cluster barrier, and the loop is bounded by max_iter.
//
// TASK = 2 (networks whose sites mostly have legs of dimension 4; blocks of 4
// warps): a warp takes the sites of a colour two at a time (positions q, q + 1
// of the colour class, which the geometry sorts by leg count); sites whose legs
// all have dimension 4 go through the half-warp pair form (both at once when
// they have the same leg count), the others through the one-site form.
// TASK = 1 (the other networks; blocks of 8 warps): one site per warp task,
// always the one-site form.  A warp visits the same sites in the same order
// every sweep: with t_slots set, their tensors are copied once into the warp's
// slots (slot_ff entries each, 16-byte aligned) and read from shared memory
// afterwards; the pair form needs them there.
template <int TASK>
__global__ void __launch_bounds__(ClusterForm<TASK>::kWarps * 32, ClusterForm<TASK>::kMinBlocks) bp_ff_cluster_kernel(BPFFParams p)
{
    constexpr int kBpClWarps = ClusterForm<TASK>::kWarps;
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(16) ff ffsmem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    ff *ws = ffsmem + wib * p.smem_per_warp;
    ff *in = ws;
    ff *out = in + kMaxDeg * kMsgStride;
    ff *u = out + kMaxDeg * kMsgStride;
    ff *w = u + p.tabA;
    ff *x1 = w + p.tabC;
    ff *x2 = x1 + p.tabA;
    const int rank = (int)cluster.block_rank(), CL = (int)cluster.num_blocks();
    const int set = blockIdx.x / CL;
    const int cwarp = rank * kBpClWarps + wib, cwarps = CL * kBpClWarps;
    const int64_t msg_set = (int64_t)p.n_legs * kMsgStride;
    ff *msg = p.msg + set * msg_set;
    const ff *Tset = p.T + set * p.set_stride;
    // with t_slots: [warps][t_slots][slot_ff] tensors, then [warps][t_slots][16]
    // current messages, then [warps][t_slots][kSlotMeta] records
    ff *tslots = nullptr, *curs = nullptr;
    int *metas = nullptr;
    if (p.t_slots > 0) {
        ff *base = ffsmem + (int64_t)kBpClWarps * p.smem_per_warp;
        tslots = base + (int64_t)wib * p.t_slots * p.slot_ff;
        base += (int64_t)kBpClWarps * p.t_slots * p.slot_ff;
        curs = base + (int64_t)wib * p.t_slots * 16;
        base += (int64_t)kBpClWarps * p.t_slots * 16;
        metas = reinterpret_cast<int *>(base) + (int64_t)wib * p.t_slots * kSlotMeta;
        int sl = 0;
        for (int ph = 0; ph < p.n_colors; ++ph) {
            const int c0 = p.color_ptr[ph], nc = p.color_ptr[ph + 1] - c0;
            for (int q = TASK * cwarp; q < nc; q += TASK * cwarps, sl += TASK)
                for (int e2 = 0; e2 < TASK && q + e2 < nc; ++e2) {
                    const int v = p.color_sites[c0 + q + e2], l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
                    const ff *src = Tset + p.tens_off[v];
                    const int n = (int)(p.tens_off[v + 1] - p.tens_off[v]);
                    ff *dst = tslots + (int64_t)(sl + e2) * p.slot_ff;
                    for (int e = lane; e < n; e += 32) dst[e] = src[e];
                    int *m = metas + (sl + e2) * kSlotMeta;
                    if (lane == 0) {
                        m[kMetaL0] = l0;
                        m[kMetaKind] = ff_pair_kind(p, v);
                        m[kMetaSite] = v;
                    }
                    if (lane < 4) m[kMetaInc + lane] = lane < k ? p.inc_slot[l0 + lane] : 0;
                    if (lane < 16 && lane / 4 < k)
                        curs[(sl + e2) * 16 + lane] = msg[(int64_t)(l0 + lane / 4) * kMsgStride + lane % 4];
                }
        }
        __syncwarp();
    }
    for (int it = 1; it <= p.max_iter; ++it) {
        // residual slots rotate over three sweeps: the slot cleared here was
        // last read before the previous sweep's barriers
        unsigned int *res_cur = p.res + (int64_t)(it % 3) * p.n_sets + set;
        if (rank == 0 && threadIdx.x == 0) p.res[(int64_t)((it + 1) % 3) * p.n_sets + set] = 0u;
        int sl = 0;
        float racc = 0.f;
        for (int ph = 0; ph < p.n_colors; ++ph) {
            const int c0 = p.color_ptr[ph], nc = p.color_ptr[ph + 1] - c0;
            for (int q = TASK * cwarp; q < nc; q += TASK * cwarps, sl += TASK) {
                const bool has_b = TASK == 2 && q + 1 < nc;
                float r;
                if constexpr (TASK == 1) {
                    const int va = metas ? metas[sl * kSlotMeta + kMetaSite] : p.color_sites[c0 + q];
                    const ff *Ta = metas ? tslots + (int64_t)sl * p.slot_ff : Tset + p.tens_off[va];
                    r = ff_site_update(p, va, Ta, msg, msg, in, out, u, w, x1, x2, lane);
                } else if (metas) {
                    const int *ma = metas + sl * kSlotMeta, *mb = has_b ? ma + kSlotMeta : ma;
                    const int ka = ma[kMetaKind], kb = has_b ? mb[kMetaKind] : 0;
                    ff *ca = curs + sl * 16, *cb = has_b ? ca + 16 : ca;
                    const ff *Ta = tslots + (int64_t)sl * p.slot_ff, *Tb = has_b ? Ta + p.slot_ff : Ta;
                    if (ka > 0 && ka == kb) {
                        const bool hi = lane >= 16;
                        r = ff_pair_dispatch(p, ka, hi ? mb : ma, hi ? cb : ca, hi ? Tb : Ta, true, msg, ws, lane);
                    } else {
                        r = ka > 0 ? ff_pair_dispatch(p, ka, ma, ca, Ta, lane < 16, msg, ws, lane)
                                   : ff_site_update(p, ma[kMetaSite], Ta, msg, msg, in, out, u, w, x1, x2, lane);
                        if (has_b)
                            r = fmaxf(r, kb > 0 ? ff_pair_dispatch(p, kb, mb, cb, Tb, lane < 16, msg, ws, lane)
                                                : ff_site_update(p, mb[kMetaSite], Tb, msg, msg, in, out, u, w, x1,
                                                                 x2, lane));
                    }
                } else {
                    const int va = p.color_sites[c0 + q];
                    r = ff_site_update(p, va, Tset + p.tens_off[va], msg, msg, in, out, u, w, x1, x2, lane);
                    if (has_b) {
                        const int vb = p.color_sites[c0 + q + 1];
                        r = fmaxf(r, ff_site_update(p, vb, Tset + p.tens_off[vb], msg, msg, in, out, u, w, x1, x2,
                                                    lane));
                    }
                }
                racc = fmaxf(racc, r);
                __syncwarp();
            }
            // one residual word per warp and sweep, before the sweep's last barrier
            if (ph + 1 == p.n_colors && lane == 0) atomicMax(res_cur, __float_as_uint(racc));
            cluster.sync();
        }
        const float rs = __uint_as_float(__ldcg(res_cur));
        if (rs < p.tol || it == p.max_iter) {
            if (rank == 0 && threadIdx.x == 0) {
                const bool conv = rs < p.tol;
                p.done_it[set] = conv ? it : 0;
                p.iters_out[set] = conv ? it : 0;
                p.res_out[set] = (double)rs;
                p.final_buf[set] = 0;
            }
            // the set's messages in FP64 for the gauge (every block of the
            // cluster wrote its share before the last barrier)
            double *m64 = p.msg64 + set * msg_set;
            for (int64_t i = (int64_t)rank * blockDim.x + threadIdx.x; i < msg_set; i += (int64_t)CL * blockDim.x) {
                const ff x = ldcg_ff(msg + i);
                m64[i] = (double)x.h + (double)x.l;
            }
            return;
        }
    }
}

// site tensors -> scaled float-float, one warp per (set, site)
// Set-up of the float-float sweeps in one launch, grid-stride: scratch words
// cleared; first messages 1/sqrt(d) as pairs; and, one warp per site, the FP64
// tensors as scaled float-float pairs -- the largest entry's exponent from the
// bits, then each entry split by integer operations (split_scaled), so the
// conversion runs at memory speed rather than on the FP64 pipe.
__global__ void ff_prepare_kernel(const double *T, ff *out, const int64_t *tens_off, int n_sites, int n_sets,
                                  int64_t stride, ff *msg, const int32_t *site_bonds, const int32_t *bond_dim,
                                  int n_legs, uint32_t *scratch, int64_t scratch_words)
{
    const int lane = threadIdx.x & 31;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < scratch_words; i += nth) scratch[i] = 0u;
    const int64_t total = (int64_t)n_sets * n_legs;
    for (int64_t i = tid; i < total; i += nth) {
        const int d = bond_dim[site_bonds[i % n_legs]];
        const double v = 1.0 / sqrt((double)d);
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - (double)hi);
        for (int a = 0; a < kMsgStride; ++a) msg[i * kMsgStride + a] = (a < d) ? ff{hi, lo} : ff{0.f, 0.f};
    }
    const int64_t items = (int64_t)n_sets * n_sites;
    for (int64_t item = tid >> 5; item < items; item += nth >> 5) {
        const int set = (int)(item / n_sites), v = (int)(item % n_sites);
        const double *t = T + set * stride + tens_off[v];
        ff *o = out + set * stride + tens_off[v];
        const int64_t n = tens_off[v + 1] - tens_off[v];
        int mxb = 0;                                     // largest biased exponent
        for (int64_t e = lane; e < n; e += 32) mxb = max(mxb, (int)((__double_as_longlong(__ldg(t + e)) >> 52) & 0x7FF));
        for (int off = 16; off > 0; off >>= 1) mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, off));
        const int ex = mxb > 0 ? min(mxb - 1022, 1022) : 0;   // entries are below 2^ex
        for (int64_t e = lane; e < n; e += 32) o[e] = split_scaled(__ldg(t + e), ex);
    }
}

// final float-float messages -> the FP64 message buffer the gauge reads
__global__ void ff_export_kernel(const ff *msg_ff, double *msg, const int32_t *final_buf, int n_sets, int64_t per_set)
{
    const int64_t total = (int64_t)n_sets * per_set;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int set = (int)(i / per_set);
        const int64_t at = ((int64_t)final_buf[set] * n_sets) * per_set + i;
        msg[at] = (double)msg_ff[at].h + (double)msg_ff[at].l;
    }
}

// ---------------------------------------------------------------- gauge
struct GaugeParams {
    int n_sets, n_bonds, n_legs;
    const int32_t *bond_site, *bond_dim, *bond_leg, *site_ptr;
    const double *msg;           // [2][n_sets][n_legs][8]
    const int32_t *final_buf;    // [n_sets]
    double *gauge;               // [n_sets][n_bonds][2][64]
    int32_t *flags;              // [1] degenerate
};

// One thread per (tensor set, bond).  With n = m0 . m1 and the Householder
// reflector H = I - 2 v v^T / (v . v) of v = m1 / |m1| + sign(m1[0]) e0, the
// gauge pair is B = [m0^T / n ; rows 1.. of H] and A = B^-1, whose column 0
// is m1 and column l >= 1 is H[l, :]^T - m1 (H[l, :] . m0) / n.  Every entry
// has a closed form in n, v and v . m0, so the FP64 work per bond is O(d^2)
// multiply-adds and three divisions.  Only the d x d corner of each 8 x 8
// slot is written; readers take no more.
__global__ void gauge_kernel(GaugeParams p)
{
    int64_t total = (int64_t)p.n_sets * p.n_bonds;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int set = (int)(i / p.n_bonds), b = (int)(i % p.n_bonds);
        double *G0 = p.gauge + (i * 2) * 64, *G1 = G0 + 64;
        const int d = p.bond_dim[b];
        const int s0 = p.bond_site[2 * b], s1 = p.bond_site[2 * b + 1];
        if (s1 < 0) {                      // open index: not partitioned
            for (int a = 0; a < d; ++a)
                for (int c = 0; c < d; ++c) { const double x = (a == c) ? 1.0 : 0.0; G0[a * 8 + c] = x; G1[a * 8 + c] = x; }
            continue;
        }
        const double *base = p.msg + ((int64_t)p.final_buf[set] * p.n_sets + set) * p.n_legs * kMsgStride;
        const double *m0p = base + (int64_t)(p.site_ptr[s0] + p.bond_leg[2 * b]) * kMsgStride;
        const double *m1p = base + (int64_t)(p.site_ptr[s1] + p.bond_leg[2 * b + 1]) * kMsgStride;
        double m0[kMaxDim], m1[kMaxDim];
#pragma unroll
        for (int a = 0; a < kMaxDim; ++a) { m0[a] = a < d ? m0p[a] : 0.0; m1[a] = a < d ? m1p[a] : 0.0; }
        double n = 0.0, nm1 = 0.0;
#pragma unroll
        for (int a = 0; a < kMaxDim; ++a) { n = fma(m0[a], m1[a], n); nm1 = fma(m1[a], m1[a], nm1); }
        if (!(fabs(n) >= 1e-300) || !(nm1 > 0.0)) { atomicExch(p.flags + 1, 1); n = 1.0; nm1 = 1.0; }
        const double inv_nm1 = 1.0 / sqrt(nm1), inv_n = 1.0 / n;
        double v[kMaxDim];
#pragma unroll
        for (int a = 0; a < kMaxDim; ++a) v[a] = m1[a] * inv_nm1;
        v[0] += (v[0] < 0.0) ? -1.0 : 1.0;
        double vv = 0.0, vm0 = 0.0;
#pragma unroll
        for (int a = 0; a < kMaxDim; ++a) { vv = fma(v[a], v[a], vv); vm0 = fma(v[a], m0[a], vm0); }
        const double k2 = 2.0 / vv;
#pragma unroll
        for (int c = 0; c < kMaxDim; ++c) {
            if (c >= d) break;
            // H[c, :] . m0 / n for the A column c (c >= 1)
            const double rc = (m0[c] - k2 * v[c] * vm0) * inv_n;
#pragma unroll
            for (int a = 0; a < kMaxDim; ++a) {
                if (a >= d) break;
                const double h = ((a == c) ? 1.0 : 0.0) - k2 * v[c] * v[a];     // H[c][a]
                G1[a * 8 + c] = (c == 0) ? m0[a] * inv_n : h;                   // B[c][a]
                G0[a * 8 + c] = (c == 0) ? m1[a] : h - m1[a] * rc;              // A[a][c]
            }
        }
    }
}


// ---------------------------------------------------------------- gauged, sliced, blocked tensors
struct BlockParams {
    int n_sets, n_slices, n_sites, n_bonds_full, n_open;
    const int32_t *open_dims;          // [n_open]
    const int32_t *open_pos;           // [n_bonds_full]: position among open bonds, or -1
    const int32_t *f_site_ptr, *f_site_bonds, *f_bond_dim, *f_bond_site;
    const int64_t *f_tens_off;
    int64_t f_stride;
    const int64_t *c_tens_off;
    int64_t c_stride;
    const int32_t *c_blk_off;          // [n_sites][64]
    const double *T;                   // [n_sets][f_stride] raw tensors
    const double *gauge;               // [n_sets][n_bonds_full][2][64]
    double *Mb;                        // [members][c_stride]
    double *z, *scale;                 // [members][n_sites]
    int8_t *zero;                      // [members][n_sites]
    int half;                          // doubles per buffer (two buffers per warp)
};

__global__ void block_kernel(BlockParams p)
{
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double *bufA = smem + (int64_t)wib * 2 * p.half;
    double *bufB = bufA + p.half;
    const int64_t members = (int64_t)p.n_sets * p.n_slices;
    const int64_t items = members * p.n_sites;
    for (int64_t item = (int64_t)blockIdx.x * wpb + wib; item < items;
         item += (int64_t)gridDim.x * wpb) {
        const int64_t member = item / p.n_sites;
        const int v = (int)(item % p.n_sites);
        const int set = (int)(member / p.n_slices), slice = (int)(member % p.n_slices);
        const int l0 = p.f_site_ptr[v], k = p.f_site_ptr[v + 1] - l0;
        int fdims[kMaxDeg], cdims[kMaxDeg], fixed[kMaxDeg], bonds[kMaxDeg], side[kMaxDeg];
        int kc = 0;
        for (int i = 0; i < k; ++i) {
            const int b = p.f_site_bonds[l0 + i];
            fdims[i] = p.f_bond_dim[b];
            bonds[i] = b;
            side[i] = (p.f_bond_site[2 * b] == v) ? 0 : 1;
            const int op = p.open_pos[b];
            if (op >= 0) {                      // slice index: row-major, last open bond fastest
                int r = slice;
                for (int q = p.n_open - 1; q > op; --q) r /= p.open_dims[q];
                fixed[i] = r % p.open_dims[op];
            } else {
                fixed[i] = -1;
                cdims[kc++] = fdims[i];
            }
        }
        int n = 1;
        for (int i = 0; i < kc; ++i) n *= cdims[i];
        // gather the slice (closed legs only) into bufA
        const double *T = p.T + set * p.f_stride + p.f_tens_off[v];
        for (int e = lane; e < n; e += 32) {
            int r = e, src = 0, mul = 1, ci = kc - 1;
            for (int i = k - 1; i >= 0; --i) {
                int dgt;
                if (fixed[i] >= 0) dgt = fixed[i];
                else { dgt = r % cdims[ci]; r /= cdims[ci]; --ci; }
                src += dgt * mul;
                mul *= fdims[i];
            }
            bufA[e] = T[src];
        }
        __syncwarp();
        // multiply each closed leg by its gauge matrix: out[.., c, ..] = sum_a in[.., a, ..] G[a][c]
        double *cur = bufA, *nxt = bufB;
        int ci = 0, post = n;
        for (int i = 0; i < k; ++i) {
            if (fixed[i] >= 0) continue;
            const int d = cdims[ci++];
            post /= d;
            const double *G = p.gauge + (((int64_t)set * p.n_bonds_full + bonds[i]) * 2 + side[i]) * 64;
            // one lane per fiber (hi, lo): its d inputs read once, its d outputs
            const int fibers = n / d;
            for (int f = lane; f < fibers; f += 32) {
                const int lo = f % post, hi = f / post;
                const int64_t base = (int64_t)hi * d * post + lo;
                double x[kMaxDim];
#pragma unroll
                for (int a = 0; a < kMaxDim; ++a) x[a] = a < d ? cur[base + (int64_t)a * post] : 0.0;
#pragma unroll
                for (int c = 0; c < kMaxDim; ++c) {
                    if (c >= d) break;
                    double s = 0.0;
#pragma unroll
                    for (int a = 0; a < kMaxDim; ++a)
                        if (a < d) s = fma(x[a], G[a * 8 + c], s);
                    nxt[base + (int64_t)c * post] = s;
                }
            }
            __syncwarp();
            double *t = cur; cur = nxt; nxt = t;
        }
        // z_v, scale, blocked write
        const double zv = cur[0];
        double mx = 0.0;
        for (int e = lane; e < n; e += 32) mx = fmax(mx, fabs(cur[e]));
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        double s;
        if (zv != 0.0) s = zv;
        else if (mx > 0.0) { int ex; frexp(mx, &ex); s = ldexp(1.0, ex); }
        else s = 1.0;
        const double inv = 1.0 / s;
        double *M = p.Mb + member * p.c_stride + p.c_tens_off[v];
        const int32_t *boff = p.c_blk_off + (int64_t)v * kBlkStride;
        for (int e = lane; e < n; e += 32) {
            int r = e, mask = 0, pos = 0, mul = 1;
            for (int i = kc - 1; i >= 0; --i) {
                const int dgt = r % cdims[i];
                r /= cdims[i];
                if (dgt > 0) { mask |= 1 << i; pos += (dgt - 1) * mul; mul *= cdims[i] - 1; }
            }
            M[boff[mask] + pos] = (zv != 0.0) ? cur[e] / zv : cur[e] * inv;
        }
        if (lane == 0) {
            p.z[member * p.n_sites + v] = zv;
            p.scale[member * p.n_sites + v] = (zv != 0.0) ? 1.0 : s;
            p.zero[member * p.n_sites + v] = (zv == 0.0) ? 1 : 0;
        }
        __syncwarp();
    }
}

// The same gauge transform and blocked write in float-float pairs on the FP32
// pipes (the partition's float-float option).  The slice is scaled by a power
// of two (its largest binary exponent, found with integer operations) before
// the split into pairs, so the pair range covers any FP64 input; the blocked
// tensor M = T' / z_v does not depend on that scale, and z_v and the scale of a
// zero site are returned to the input's scale exactly.
__global__ void block_ff_kernel(BlockParams p)
{
    extern __shared__ double smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    ff *bufA = reinterpret_cast<ff *>(smem + (int64_t)wib * 2 * p.half);
    ff *bufB = bufA + p.half;
    ff *Gs = reinterpret_cast<ff *>(smem + (int64_t)wpb * 2 * p.half) + wib * 64;   // one leg's gauge matrix
    const int64_t members = (int64_t)p.n_sets * p.n_slices;
    const int64_t items = members * p.n_sites;
    for (int64_t item = (int64_t)blockIdx.x * wpb + wib; item < items;
         item += (int64_t)gridDim.x * wpb) {
        const int64_t member = item / p.n_sites;
        const int v = (int)(item % p.n_sites);
        const int set = (int)(member / p.n_slices), slice = (int)(member % p.n_slices);
        const int l0 = p.f_site_ptr[v], k = p.f_site_ptr[v + 1] - l0;
        int cdims[kMaxDeg], bonds[kMaxDeg], side[kMaxDeg], cstr[kMaxDeg];
        float cinv[kMaxDeg];
        int kc = 0, fixed_off = 0, mul = 1;
        // strides of the closed legs in the raw tensor, and the offset of the
        // fixed open-leg digits of this slice
        for (int i = k - 1; i >= 0; --i) {
            const int b = p.f_site_bonds[l0 + i];
            const int d = p.f_bond_dim[b];
            const int op = p.open_pos[b];
            if (op >= 0) {
                int r = slice;
                for (int q = p.n_open - 1; q > op; --q) r /= p.open_dims[q];
                fixed_off += (r % p.open_dims[op]) * mul;
            } else {
                ++kc;
            }
            mul *= d;
        }
        {
            int ci = kc, m2 = 1;
            for (int i = k - 1; i >= 0; --i) {
                const int b = p.f_site_bonds[l0 + i];
                const int d = p.f_bond_dim[b];
                if (p.open_pos[b] < 0) {
                    --ci;
                    cdims[ci] = d; cinv[ci] = 1.0f / (float)d; cstr[ci] = m2;
                    bonds[ci] = b; side[ci] = (p.f_bond_site[2 * b] == v) ? 0 : 1;
                }
                m2 *= d;
            }
        }
        int n = 1;
        for (int i = 0; i < kc; ++i) n *= cdims[i];
        const double *T = p.T + set * p.f_stride + p.f_tens_off[v] + fixed_off;
        const bool ident = kc == k;          // no open legs: the slice is the tensor itself
        auto src_of = [&](int e) {
            if (ident) return e;
            int r = e, src = 0;
            for (int i = kc - 1; i >= 0; --i) { int dgt; r = fdivmod(r, cdims[i], cinv[i], dgt); src += dgt * cstr[i]; }
            return src;
        };
        // largest biased exponent of the slice, then the scaled pairs
        int mxb = 0;
        for (int e = lane; e < n; e += 32)
            mxb = max(mxb, (int)((__double_as_longlong(T[src_of(e)]) >> 52) & 0x7FF));
        for (int off = 16; off > 0; off >>= 1) mxb = max(mxb, __shfl_xor_sync(0xffffffffu, mxb, off));
        const int ex = mxb > 0 ? min(mxb - 1022, 1022) : 0;        // slice values are below 2^ex
        for (int e = lane; e < n; e += 32) bufA[e] = split_scaled(T[src_of(e)], ex);
        __syncwarp();
        ff *cur = bufA, *nxt = bufB;
        int post = n;
        for (int i = 0; i < kc; ++i) {
            const int d = cdims[i];
            post /= d;
            const double *G = p.gauge + (((int64_t)set * p.n_bonds_full + bonds[i]) * 2 + side[i]) * 64;
            for (int q = lane; q < d * 8; q += 32)
                if ((q & 7) < d) Gs[q] = split_scaled(G[q], 0);
            __syncwarp();
            // one lane per fiber (hi, lo) of this leg: its d inputs are read
            // once and give its d outputs, each summed over a in order
            const float inv_post = 1.0f / (float)post;
            const int fibers = n / d;
            for (int f = lane; f < fibers; f += 32) {
                int lo;
                const int hi = fdivmod(f, post, inv_post, lo);
                const int64_t base = (int64_t)hi * d * post + lo;
                ff x[kMaxDim];
#pragma unroll
                for (int a = 0; a < kMaxDim; ++a) x[a] = a < d ? cur[base + (int64_t)a * post] : ff{0.f, 0.f};
#pragma unroll
                for (int c = 0; c < kMaxDim; ++c) {
                    if (c >= d) break;
                    ffacc acc;
#pragma unroll
                    for (int a = 0; a < kMaxDim; ++a)
                        if (a < d) acc.mad(x[a], Gs[a * 8 + c]);
                    nxt[base + (int64_t)c * post] = acc.get();
                }
            }
            __syncwarp();
            ff *t = cur; cur = nxt; nxt = t;
        }
        // z_v, scale, blocked write (in the slice's scale, returned to the input's)
        const ff zv = cur[0];
        const bool zero_site = (zv.h == 0.f);
        int mob = 0;
        for (int e = lane; e < n; e += 32) mob = max(mob, (__float_as_int(cur[e].h) >> 23) & 0xFF);
        for (int off = 16; off > 0; off >>= 1) mob = max(mob, __shfl_xor_sync(0xffffffffu, mob, off));
        // scale of a zero site: 2^e with e the frexp exponent of its largest entry
        const int se = mob > 0 ? mob - 126 : 0;
        const ff inv_s = {__int_as_float((127 - se) << 23), 0.f};   // 2^-se
        double *M = p.Mb + member * p.c_stride + p.c_tens_off[v];
        const int32_t *boff = p.c_blk_off + (int64_t)v * kBlkStride;
        const ff f = zero_site ? inv_s : ff_div({1.f, 0.f}, zv);
        for (int e = lane; e < n; e += 32) {
            int r = e, mask = 0, pos = 0, bm = 1;
            for (int i = kc - 1; i >= 0; --i) {
                int dgt;
                r = fdivmod(r, cdims[i], cinv[i], dgt);
                if (dgt > 0) { mask |= 1 << i; pos += (dgt - 1) * bm; bm *= cdims[i] - 1; }
            }
            const ff m = ff_mul(cur[e], f);
            M[boff[mask] + pos] = widen(m.h) + widen(m.l);
        }
        if (lane == 0) {
            const double up = __longlong_as_double((long long)(1023 + ex) << 52);   // 2^ex
            const double zt = ((double)zv.h + (double)zv.l) * up;
            p.z[member * p.n_sites + v] = zt;
            p.scale[member * p.n_sites + v] = zero_site ? ldexp(1.0, se) * up : 1.0;
            p.zero[member * p.n_sites + v] = zero_site ? 1 : 0;
        }
        __syncwarp();
    }
}

// ln|Z_ref|, sign(Z_ref) and the number of zero sites, one block per member:
// per-thread partials over a fixed stride, then a fixed shared-memory tree, so
// the sum order depends only on the site count.  (The FP64 logarithm is long;
// a block per member spreads it over the SMs.)
constexpr int kVacThreads = 256;

__global__ void __launch_bounds__(kVacThreads) vacuum_kernel(const double *z, int n_sites, int64_t members, double *vac)
{
    __shared__ double s_lg[kVacThreads];
    __shared__ int s_neg[kVacThreads], s_nz[kVacThreads];
    const int64_t m = blockIdx.x;
    if (m >= members) return;
    double lg = 0.0;
    int neg = 0, nz = 0;
    for (int v = threadIdx.x; v < n_sites; v += kVacThreads) {
        const double x = z[m * n_sites + v];
        if (x == 0.0) { ++nz; continue; }
        lg += log(fabs(x));
        neg += (x < 0.0);
    }
    s_lg[threadIdx.x] = lg; s_neg[threadIdx.x] = neg; s_nz[threadIdx.x] = nz;
    __syncthreads();
    for (int h = kVacThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) {
            s_lg[threadIdx.x] += s_lg[threadIdx.x + h];
            s_neg[threadIdx.x] += s_neg[threadIdx.x + h];
            s_nz[threadIdx.x] += s_nz[threadIdx.x + h];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        vac[3 * m] = s_lg[0];
        vac[3 * m + 1] = (s_neg[0] & 1) ? -1.0 : 1.0;
        vac[3 * m + 2] = (double)s_nz[0];
    }
}

__device__ __forceinline__ float round_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__global__ void convert_kernel(const double *src, int64_t n, int dtype, float *dst32, __nv_bfloat16 *dst16)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float f = (float)src[i];
        if (dtype == PNE_BF16) dst16[i] = __float2bfloat16_rn(f);
        else dst32[i] = (dtype == PNE_TF32) ? round_tf32(f) : f;
    }
}

int grid_for(int64_t n, int block, int n_sm)
{
    int64_t g = (n + block - 1) / block;
    int64_t cap = (int64_t)n_sm * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ---------------------------------------------------------------- host launchers
namespace {

// Raises a kernel's dynamic shared-memory limit (process-wide, only upwards).
template <typename F>
void grant_smem(pne_ctx *ctx, int slot, F func, size_t bytes)
{
    (void)ctx; (void)slot;
    grant_dynamic_smem((const void *)func, bytes);
}

}  // namespace

pne_status launch_bp(pne_ctx *ctx, pne_partition *p, double tol, int max_iter, double damping,
                     cudaStream_t s, void *rec, int arithmetic, cudaMemcpyKind rec_kind)
{
    HostScope hs__(ctx, "part_bp");
    const Geometry &g = p->geo->full;
    const int n_sets = p->n_sets;
    // table sizes: halves of the largest site
    int tabA = 1, tabC = 1;
    for (int v = 0; v < g.n_sites; ++v) {
        const int k = g.site_ptr[v + 1] - g.site_ptr[v], h = k / 2;
        int A = 1, C = 1;
        for (int i = 0; i < k; ++i) {
            const int d = g.bond_dim[g.site_bonds[g.site_ptr[v] + i]];
            if (i < h) A *= d; else C *= d;
        }
        tabA = tabA > A ? tabA : A;
        tabC = tabC > C ? tabC : C;
    }
    const int per_warp = 2 * kMaxDeg * kMsgStride + 2 * tabA + 2 * tabC;
    const size_t smem = (size_t)per_warp * kBpWarps * sizeof(double);
    if (smem > 200 * 1024) {
        set_error(ctx, PNE_EINVAL, "site tensor too large for the BP kernel");
        return PNE_EINVAL;
    }
    // scratch: res[4][n_sets] u64, then the convergence record as it is read
    // back -- res_out [n_sets] f64, flags[4] i32, iters [n_sets] i32 -- then
    // done/final [n_sets] i32, barrier[2] u32; in float-float arithmetic the
    // pair tensors and pair messages follow (one allocation)
    const size_t rec_bytes = (size_t)n_sets * 12 + 16;
    const size_t bytes = ((4 * n_sets * 8 + rec_bytes + 2 * n_sets * 4 + 8) + 255) & ~size_t(255);
    const int64_t stride = g.tens_off[g.n_sites];
    const size_t tbytes = arithmetic == 1 ? (size_t)n_sets * stride * sizeof(ff) : 0;
    const size_t mbytes = arithmetic == 1 ? (size_t)2 * n_sets * g.n_legs * kMsgStride * sizeof(ff) : 0;
    DevBuf scratch;
    pne_status st = dev_alloc(ctx, scratch, bytes + tbytes + mbytes, s);
    if (st) return st;
    char *base = (char *)scratch.ptr;
    unsigned long long *res = (unsigned long long *)base;
    char *rec_dev = base + 4 * n_sets * 8;
    double *res_out = (double *)rec_dev;
    int32_t *flags = (int32_t *)(rec_dev + n_sets * 8);
    int32_t *iters = flags + 4;
    int32_t *done = iters + n_sets;
    int32_t *finalb = done + n_sets;
    unsigned int *bar = (unsigned int *)(finalb + n_sets);
    cudaError_t e;

    double *msg = (double *)p->msg.ptr;
    if (arithmetic == 1) {
        // float-float sweeps: pair tensors and pair messages after the
        // scratch words, the final messages exported to the FP64 buffer for
        // the gauge; one launch converts the tensors, sets the first messages
        // and clears the scratch words
        ff *Tff = (ff *)(base + bytes);
        ff *mff = (ff *)(base + bytes + tbytes);
        {
            ProfScope ps(ctx, s, "bp_init");
            const int64_t warps = (int64_t)n_sets * g.n_sites;
            ff_prepare_kernel<<<grid_for(warps * 32, 256, ctx->n_sm), 256, 0, s>>>(
                (const double *)p->T.ptr, Tff, g.d_tens_off, g.n_sites, n_sets, stride, mff, g.d_site_bonds,
                g.d_bond_dim, g.n_legs, (uint32_t *)base, (int64_t)(bytes / 4));
        }
        // the sweeps read what this launch writes (pair tensors, first
        // messages, cleared scratch words): it must have been queued
        if (cudaGetLastError() != cudaSuccess) {
            dev_free(ctx, scratch, s);
            set_error(ctx, PNE_ECUDA, "ff_prepare_kernel launch failed");
            return PNE_ECUDA;
        }
        BPFFParams fp;
        fp.n_sets = n_sets; fp.n_sites = g.n_sites; fp.n_legs = g.n_legs;
        fp.site_ptr = g.d_site_ptr; fp.site_bonds = g.d_site_bonds; fp.bond_dim = g.d_bond_dim;
        fp.inc_slot = g.d_inc_slot; fp.tens_off = g.d_tens_off; fp.set_stride = stride;
        fp.T = Tff; fp.msg = mff; fp.tol = (float)tol; fp.damping = damping; fp.max_iter = max_iter;
        fp.res = (unsigned int *)res; fp.done_it = done; fp.iters_out = iters; fp.final_buf = finalb;
        fp.flags = flags; fp.res_out = res_out; fp.bar = bar;
        fp.smem_per_warp = per_warp; fp.tabA = tabA; fp.tabC = tabC;
        fp.n_colors = g.n_colors; fp.color_ptr = g.d_color_ptr; fp.color_sites = g.d_color_sites;
        fp.msg64 = msg;
        // one cluster per tensor set when the colour classes are small enough
        // (at most four warp tasks per warp and phase in a cluster of <= 16
        // blocks); two sites per task when at least half of the sites take
        // the pair form (every leg of dimension 4, 2 to 4 legs)
        int max_color = 0;
        for (int c = 0; c < g.n_colors; ++c) max_color = std::max(max_color, g.color_ptr[c + 1] - g.color_ptr[c]);
        int n_pair = 0;
        for (int v = 0; v < g.n_sites; ++v) {
            const int k = g.site_ptr[v + 1] - g.site_ptr[v];
            bool all4 = k >= 2 && k <= 4;
            for (int i = 0; i < k && all4; ++i) all4 = g.bond_dim[g.site_bonds[g.site_ptr[v] + i]] == 4;
            n_pair += all4 ? 1 : 0;
        }
        // the cluster form's warp scratch also holds the pair form's (128 ff)
        const int per_warp_cl = std::max(per_warp, 128);
        int slot_ff = 0;
        for (int v = 0; v < g.n_sites; ++v)
            slot_ff = std::max<int>(slot_ff, (int)(g.tens_off[v + 1] - g.tens_off[v]));
        slot_ff = (slot_ff + 1) & ~1;
        // per slot: the tensor, the current messages [4][4], the record
        const size_t slot_bytes = (size_t)slot_ff * sizeof(ff) + 16 * sizeof(ff) + kSlotMeta * sizeof(int);
        // slots per warp for `task` sites per warp task, `warps` warps per
        // block and a cluster of cl blocks (a warp takes ceil(ceil(nc / task) /
        // (cl warps)) tasks of each colour), kept only while the block's shared
        // memory stays within kBpTensorSmem
        auto slots_of = [&](int task_, int warps, int cl) {
            int n = 0;
            for (int c = 0; c < g.n_colors; ++c) {
                const int tasks = (g.color_ptr[c + 1] - g.color_ptr[c] + task_ - 1) / task_;
                n += task_ * ((tasks + cl * warps - 1) / (cl * warps));
            }
            const size_t b = (size_t)per_warp_cl * warps * sizeof(double) + (size_t)warps * n * slot_bytes;
            return b <= kBpTensorSmem ? n : 0;
        };
        auto cluster_for = [&](int task_, int warps) {
            int cl = 1;
            while (cl * warps * task_ < max_color && cl < 16) cl *= 2;
            return cl;
        };
        // the pair form needs the site tensors in shared memory
        const int task = (2 * n_pair >= g.n_sites &&
                          slots_of(2, ClusterForm<2>::kWarps, cluster_for(2, ClusterForm<2>::kWarps)) > 0) ? 2 : 1;
        const int kBpClWarps = task == 2 ? ClusterForm<2>::kWarps : ClusterForm<1>::kWarps;
        const void *cl_kernel = task == 2 ? (const void *)bp_ff_cluster_kernel<2> : (const void *)bp_ff_cluster_kernel<1>;
        int CL = cluster_for(task, kBpClWarps);
        bool cluster_ok = g.n_colors > 0 && max_color <= CL * kBpClWarps * task * 4;
        const size_t smem_cl = (size_t)per_warp_cl * kBpClWarps * sizeof(double);
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute cattr[1];
        fp.t_slots = 0;
        fp.slot_ff = 0;
        if (cluster_ok) {
            auto slots_for = [&](int cl) { return slots_of(task, kBpClWarps, cl); };
            auto smem_for = [&](int cl) { return smem_cl + (size_t)kBpClWarps * slots_for(cl) * slot_bytes; };
            cfg.blockDim = dim3(kBpClWarps * 32);
            cfg.stream = s;
            cattr[0].id = cudaLaunchAttributeClusterDimension;
            cattr[0].val.clusterDim.y = 1;
            cattr[0].val.clusterDim.z = 1;
            cfg.attrs = cattr;
            cfg.numAttrs = 1;
            // the largest cluster the device schedules with this kernel's
            // resources; whether (shared memory, cluster size) fits is queried
            // once per context
            int chosen = 0;
            for (int cl = CL;;) {
                const size_t sm = smem_for(cl);
                const std::pair<size_t, int> key{sm, cl + 64 * task};
                int fits = -1;
                {
                    std::lock_guard<std::mutex> lk(ctx->launch_mu);
                    auto it = ctx->bp_cluster.find(key);
                    if (it != ctx->bp_cluster.end()) fits = it->second;
                }
                if (fits < 0) {
                    grant_dynamic_smem(cl_kernel, sm);
                    cudaFuncSetAttribute(cl_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
                    cattr[0].val.clusterDim.x = cl;
                    cfg.gridDim = dim3(cl);
                    cfg.dynamicSmemBytes = sm;
                    int ncl = 0;
                    fits = (cudaOccupancyMaxActiveClusters(&ncl, cl_kernel, &cfg) == cudaSuccess &&
                            ncl > 0) ? 1 : 0;
                    cudaGetLastError();
                    std::lock_guard<std::mutex> lk(ctx->launch_mu);
                    ctx->bp_cluster[key] = fits;
                }
                if (fits) { chosen = cl; break; }
                if (cl == 1) break;
                cl /= 2;
                if (max_color > cl * kBpClWarps * task * 4) break;
            }
            if (chosen > 0) {
                CL = chosen;
                cattr[0].val.clusterDim.x = CL;
                cfg.dynamicSmemBytes = smem_for(CL);
                grant_dynamic_smem(cl_kernel, cfg.dynamicSmemBytes);
                fp.t_slots = slots_for(CL);
                fp.slot_ff = fp.t_slots > 0 ? slot_ff : 0;
                fp.smem_per_warp = per_warp_cl;
            } else {
                cluster_ok = false;
            }
        }
        int nb_ff = 1;
        if (!cluster_ok) {
            grant_smem(ctx, 1, bp_ff_kernel, smem);
            int per_sm_ff = 0;
            {
                std::lock_guard<std::mutex> lk(ctx->launch_mu);
                auto it = ctx->bp_grid_occ.find(smem);
                if (it != ctx->bp_grid_occ.end()) per_sm_ff = it->second;
            }
            if (per_sm_ff == 0) {
                PNE_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_ff, bp_ff_kernel, kBpWarps * 32, smem));
                std::lock_guard<std::mutex> lk(ctx->launch_mu);
                ctx->bp_grid_occ[smem] = per_sm_ff;
            }
            if (per_sm_ff < 1) { dev_free(ctx, scratch, s); set_error(ctx, PNE_EINVAL, "BP kernel does not fit"); return PNE_EINVAL; }
            const int64_t items_ff = (int64_t)n_sets * g.n_sites;
            const int64_t want_ff = (items_ff + kBpWarps - 1) / kBpWarps, cap_ff = (int64_t)per_sm_ff * ctx->n_sm;
            nb_ff = (int)std::max<int64_t>(1, want_ff < cap_ff ? want_ff : cap_ff);
        }
        void *fargs[] = {&fp};
        cudaError_t fe;
        {
            ProfScope ps(ctx, s, "bp_sweeps");
            if (cluster_ok) {
                cfg.gridDim = dim3((unsigned)(n_sets * CL));
                fe = task == 2 ? cudaLaunchKernelEx(&cfg, bp_ff_cluster_kernel<2>, fp)
                               : cudaLaunchKernelEx(&cfg, bp_ff_cluster_kernel<1>, fp);
            } else {
                fe = cudaLaunchCooperativeKernel((void *)bp_ff_kernel, dim3(nb_ff), dim3(kBpWarps * 32), fargs, smem, s);
            }
        }
        if (fe != cudaSuccess) { dev_free(ctx, scratch, s); PNE_CUDA_TRY(ctx, fe); }
        if (!cluster_ok) {
            // the cluster form writes the FP64 messages itself as it stops
            ProfScope ps(ctx, s, "bp_export");
            ff_export_kernel<<<grid_for((int64_t)n_sets * g.n_legs * kMsgStride, 256, ctx->n_sm), 256, 0, s>>>(
                mff, msg, finalb, n_sets, (int64_t)g.n_legs * kMsgStride);
        }
        PNE_CUDA_TRY(ctx, cudaGetLastError());
    }
    if (arithmetic != 1) {
    e = cudaMemsetAsync(scratch.ptr, 0, bytes, s);
    if (e != cudaSuccess) { dev_free(ctx, scratch, s); PNE_CUDA_TRY(ctx, e); }
    {
        ProfScope ps(ctx, s, "bp_init");
        bp_init_kernel<<<grid_for((int64_t)n_sets * g.n_legs, 256, ctx->n_sm), 256, 0, s>>>(
            msg, g.d_site_ptr, g.d_site_bonds, g.d_bond_dim, g.n_sites, g.n_legs, n_sets);
    }
    if (cudaGetLastError() != cudaSuccess) {
        dev_free(ctx, scratch, s);
        set_error(ctx, PNE_ECUDA, "bp_init_kernel launch failed");
        return PNE_ECUDA;
    }

    BPParams prm;
    prm.n_sets = n_sets; prm.n_sites = g.n_sites; prm.n_legs = g.n_legs;
    prm.site_ptr = g.d_site_ptr; prm.site_bonds = g.d_site_bonds; prm.bond_dim = g.d_bond_dim;
    prm.inc_slot = g.d_inc_slot; prm.tens_off = g.d_tens_off; prm.set_stride = g.tens_off[g.n_sites];
    prm.T = (const double *)p->T.ptr; prm.msg = msg;
    prm.tol = tol; prm.damping = damping; prm.max_iter = max_iter;
    prm.res = res; prm.done_it = done; prm.iters_out = iters; prm.res_out = res_out;
    prm.final_buf = finalb; prm.flags = flags; prm.bar = bar;
    prm.smem_per_warp = per_warp; prm.tabA = tabA; prm.tabC = tabC;
    prm.n_colors = g.n_colors; prm.color_ptr = g.d_color_ptr; prm.color_sites = g.d_color_sites;

    grant_smem(ctx, 2, bp_persistent_kernel, smem);
    int per_sm = 0;
    PNE_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bp_persistent_kernel,
                                                                     kBpWarps * 32, smem));
    if (per_sm < 1) { dev_free(ctx, scratch, s); set_error(ctx, PNE_EINVAL, "BP kernel does not fit"); return PNE_EINVAL; }
    const int64_t items = (int64_t)n_sets * g.n_sites;
    int64_t want = (items + kBpWarps - 1) / kBpWarps;
    int64_t cap = (int64_t)per_sm * ctx->n_sm;
    int nblocks = (int)(want < cap ? want : cap);
    if (nblocks < 1) nblocks = 1;
    void *args[] = {&prm};
    {
        ProfScope ps(ctx, s, "bp_sweeps");
        e = cudaLaunchCooperativeKernel((void *)bp_persistent_kernel, dim3(nblocks), dim3(kBpWarps * 32),
                                        args, smem, s);
    }
    if (e != cudaSuccess) { dev_free(ctx, scratch, s); PNE_CUDA_TRY(ctx, e); }
    }
    // the final-buffer index stays on the device for the gauge kernel
    if (p->gauge.ptr == nullptr) { dev_free(ctx, scratch, s); return PNE_EINVAL; }
    GaugeParams gp;
    gp.n_sets = n_sets; gp.n_bonds = g.n_bonds; gp.n_legs = g.n_legs;
    gp.bond_site = g.d_bond_site; gp.bond_dim = g.d_bond_dim; gp.bond_leg = g.d_bond_leg;
    gp.site_ptr = g.d_site_ptr; gp.msg = msg; gp.final_buf = finalb;
    gp.gauge = (double *)p->gauge.ptr; gp.flags = flags;
    {
        ProfScope ps(ctx, s, "gauge");
        gauge_kernel<<<grid_for((int64_t)n_sets * g.n_bonds, 128, ctx->n_sm), 128, 0, s>>>(gp);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    // the convergence record (residuals, flags of BP and the gauge, sweeps) in one copy
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(rec, rec_dev, rec_bytes, rec_kind, s));
    dev_free(ctx, scratch, s);
    return PNE_OK;
}

// user projectors: closed bond b = (s0, s1) takes u_b as the message on s1's
// leg (the vector that arrives at s0) and v_b on s0's leg, which is the rank-1
// projector P_b = u_b v_b^T / (u_b . v_b) of the gauge below (buffer 0)
__global__ void user_proj_kernel(const double *u, const double *v, const int64_t *off, int64_t per_set, int n_sets,
                                 int n_bonds, int n_legs, const int32_t *bond_site, const int32_t *bond_dim,
                                 const int32_t *bond_leg, const int32_t *site_ptr, double *msg)
{
    const int64_t total = (int64_t)n_sets * n_bonds * kMsgStride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int a = (int)(i % kMsgStride);
        const int b = (int)((i / kMsgStride) % n_bonds), set = (int)(i / ((int64_t)kMsgStride * n_bonds));
        const int s0 = bond_site[2 * b], s1 = bond_site[2 * b + 1];
        if (s1 < 0 || a >= bond_dim[b]) continue;
        double *base = msg + (int64_t)set * n_legs * kMsgStride;
        const int64_t src = (int64_t)set * per_set + off[b] + a;
        base[(int64_t)(site_ptr[s1] + bond_leg[2 * b + 1]) * kMsgStride + a] = u[src];
        base[(int64_t)(site_ptr[s0] + bond_leg[2 * b]) * kMsgStride + a] = v[src];
    }
}

pne_status launch_user_projectors(pne_ctx *ctx, pne_partition *p, const double *user_u, const double *user_v,
                                  cudaStream_t s, void *rec, cudaMemcpyKind rec_kind)
{
    HostScope hs__(ctx, "part_user_proj");
    const Geometry &g = p->geo->full;
    const int n_sets = p->n_sets;
    std::vector<int64_t> off(std::max(g.n_bonds, 1), -1);
    int64_t per_set = 0;
    for (int b = 0; b < g.n_bonds; ++b)
        if (g.bond_site[2 * b + 1] >= 0) { off[b] = per_set; per_set += g.bond_dim[b]; }
    // scratch: the record (residuals [n_sets] f64, flags[4] i32, sweeps [n_sets]
    // i32, all zero but the gauge's degenerate flag), final buffers [n_sets]
    // i32 (0), then the bond offsets and the two vector arrays
    const size_t rec_bytes = (size_t)n_sets * 12 + 16;
    const size_t head = ((rec_bytes + (size_t)n_sets * 4) + 255) & ~size_t(255);
    const size_t off_bytes = ((size_t)off.size() * 8 + 255) & ~size_t(255);
    const size_t vec_bytes = (size_t)n_sets * per_set * 8;
    DevBuf scratch;
    pne_status st = dev_alloc(ctx, scratch, head + off_bytes + 2 * std::max<size_t>(vec_bytes, 8), s);
    if (st) return st;
    char *base = (char *)scratch.ptr;
    int32_t *flags = (int32_t *)(base + (size_t)n_sets * 8);
    int32_t *finalb = (int32_t *)(base + rec_bytes);
    int64_t *d_off = (int64_t *)(base + head);
    double *d_u = (double *)(base + head + off_bytes), *d_v = d_u + std::max<int64_t>((int64_t)n_sets * per_set, 1);
    auto fail = [&](pne_status e) { dev_free(ctx, scratch, s); return e; };
    if (cudaMemsetAsync(base, 0, head, s) != cudaSuccess) return fail(PNE_ECUDA);
    if ((st = upload(ctx, d_off, off.data(), off.size() * 8, s))) return fail(st);
    if (vec_bytes && ((st = upload(ctx, d_u, user_u, vec_bytes, s)) || (st = upload(ctx, d_v, user_v, vec_bytes, s))))
        return fail(st);
    double *msg = (double *)p->msg.ptr;
    {
        ProfScope ps(ctx, s, "bp_init");
        user_proj_kernel<<<grid_for((int64_t)n_sets * g.n_bonds * kMsgStride, 256, ctx->n_sm), 256, 0, s>>>(
            d_u, d_v, d_off, per_set, n_sets, g.n_bonds, g.n_legs, g.d_bond_site, g.d_bond_dim, g.d_bond_leg,
            g.d_site_ptr, msg);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(PNE_ECUDA);
    GaugeParams gp;
    gp.n_sets = n_sets; gp.n_bonds = g.n_bonds; gp.n_legs = g.n_legs;
    gp.bond_site = g.d_bond_site; gp.bond_dim = g.d_bond_dim; gp.bond_leg = g.d_bond_leg;
    gp.site_ptr = g.d_site_ptr; gp.msg = msg; gp.final_buf = finalb;
    gp.gauge = (double *)p->gauge.ptr; gp.flags = flags;
    {
        ProfScope ps(ctx, s, "gauge");
        gauge_kernel<<<grid_for((int64_t)n_sets * g.n_bonds, 128, ctx->n_sm), 128, 0, s>>>(gp);
    }
    if (cudaGetLastError() != cudaSuccess) return fail(PNE_ECUDA);
    if (cudaMemcpyAsync(rec, base, rec_bytes, rec_kind, s) != cudaSuccess) return fail(PNE_ECUDA);
    dev_free(ctx, scratch, s);
    return PNE_OK;
}

pne_status launch_gauge(pne_ctx *ctx, pne_partition *p, cudaStream_t s, int32_t *h_flag)
{
    HostScope hs__(ctx, "part_gauge");
    (void)h_flag;
    const Geometry &f = p->geo->full, &c = p->geo->closed;
    const int nmax = p->geo->gauge_nmax;
    if (nmax > 4096) { set_error(ctx, PNE_EINVAL, "site tensor larger than 4096 entries"); return PNE_EINVAL; }
    const int half = nmax < 32 ? 32 : nmax;
    int wpb = (int)((48 * 1024) / (2 * half * sizeof(double)));
    if (wpb > 8) wpb = 8;
    if (wpb < 1) wpb = 1;
    const size_t smem = (size_t)wpb * 2 * half * sizeof(double);
    // geometry table of open positions and dims (built with the geometry)
    const int32_t *d_open_pos = (const int32_t *)p->geo->gauge_tab.ptr, *d_open_dims = d_open_pos + f.n_bonds;
    BlockParams bp;
    bp.n_sets = p->n_sets; bp.n_slices = p->n_slices; bp.n_sites = f.n_sites;
    bp.n_bonds_full = f.n_bonds; bp.n_open = (int)p->geo->open_bonds.size();
    bp.open_dims = d_open_dims; bp.open_pos = d_open_pos;
    bp.f_site_ptr = f.d_site_ptr; bp.f_site_bonds = f.d_site_bonds; bp.f_bond_dim = f.d_bond_dim;
    bp.f_bond_site = f.d_bond_site; bp.f_tens_off = f.d_tens_off; bp.f_stride = f.tens_off[f.n_sites];
    bp.c_tens_off = c.d_tens_off; bp.c_stride = c.tens_off[c.n_sites]; bp.c_blk_off = c.d_blk_off;
    bp.T = (const double *)p->T.ptr; bp.gauge = (const double *)p->gauge.ptr;
    bp.Mb = (double *)p->Mb.ptr;
    bp.z = (double *)p->site_info.ptr; bp.scale = (double *)p->site_scale.ptr;
    bp.zero = (int8_t *)p->site_zero.ptr;
    bp.half = half;
    const int64_t items = (int64_t)p->n_members * f.n_sites;
    int64_t g = (items + wpb - 1) / wpb;
    if (g > (int64_t)ctx->n_sm * 16) g = (int64_t)ctx->n_sm * 16;
    {
        ProfScope ps(ctx, s, "gauge_block");
        if (p->arithmetic == 1) {
            const size_t smem_ff = smem + (size_t)wpb * 64 * sizeof(ff);   // plus one gauge matrix per warp
            grant_smem(ctx, 3, block_ff_kernel, smem_ff);
            block_ff_kernel<<<(int)g, wpb * 32, smem_ff, s>>>(bp);
        } else {
            grant_smem(ctx, 4, block_kernel, smem);
            block_kernel<<<(int)g, wpb * 32, smem, s>>>(bp);
        }
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    {
        ProfScope ps(ctx, s, "vacuum");
        vacuum_kernel<<<(unsigned)p->n_members, kVacThreads, 0, s>>>((const double *)p->site_info.ptr, f.n_sites,
                                                                    p->n_members, (double *)p->vac.ptr);
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}

pne_status convert_buffer(pne_ctx *ctx, const double *src, int64_t n, int dtype, void *dst, cudaStream_t s)
{
    if (dtype == PNE_BF16)
        convert_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>(src, n, dtype, nullptr, (__nv_bfloat16 *)dst);
    else
        convert_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>(src, n, dtype, (float *)dst, nullptr);
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}

// conversion only, into buffers that already exist (safe inside stream capture)
pne_status launch_convert_only(pne_ctx *ctx, const pne_partition *p, int dtype, cudaStream_t s)
{
    if (dtype == PNE_F64) return PNE_OK;
    const int64_t n = (int64_t)p->n_members * p->geo->closed.tens_off[p->geo->closed.n_sites];
    ProfScope ps(ctx, s, "convert");
    if (dtype == PNE_BF16)
        convert_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>((const double *)p->Mb.ptr, n, dtype, nullptr,
                                                                   (__nv_bfloat16 *)p->Mb16.ptr);
    else
        convert_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>((const double *)p->Mb.ptr, n, dtype,
                                                                   (float *)p->Mb32.ptr, nullptr);
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}

pne_status launch_convert(pne_ctx *ctx, pne_partition *p, int dtype, cudaStream_t s)
{
    if (dtype == PNE_F64 || p->mb32_dtype == dtype) return PNE_OK;
    const int64_t n = (int64_t)p->n_members * p->geo->closed.tens_off[p->geo->closed.n_sites];
    pne_status st;
    if (dtype == PNE_BF16) {
        if (!p->Mb16.ptr && (st = dev_alloc(ctx, p->Mb16, n * 2, s))) return st;
        ProfScope ps(ctx, s, "convert");
        convert_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>(
            (const double *)p->Mb.ptr, n, dtype, nullptr, (__nv_bfloat16 *)p->Mb16.ptr);
    } else {
        if (!p->Mb32.ptr && (st = dev_alloc(ctx, p->Mb32, n * 4, s))) return st;
        ProfScope ps(ctx, s, "convert");
        convert_kernel<<<grid_for(n, 256, ctx->n_sm), 256, 0, s>>>(
            (const double *)p->Mb.ptr, n, dtype, (float *)p->Mb32.ptr, nullptr);
        p->mb32_dtype = dtype;
    }
    PNE_CUDA_TRY(ctx, cudaGetLastError());
    return PNE_OK;
}

}  // namespace pne

// ---------------------------------------------------------------- BP without device allocation
// Working memory of pne_bp_messages_noalloc: one file-scope device array.
// Host code only ever passes its device address (looked up per device).
static __device__ __align__(256) unsigned char g_bp_noalloc_scratch[PNE_NOALLOC_SCRATCH_BYTES];

namespace pne {
namespace {

constexpr int kNoAllocMaxDevices = 64;
// device address of the array, per device (host threads may race to fill an
// entry; each writes the same address)
std::atomic<void *> g_noalloc_addr[kNoAllocMaxDevices] = {};

// bond_leg, incoming-message slots and tensor offsets from the raw geometry,
// one thread (tables are small; the call allocates nothing to go faster)
__global__ void noalloc_tables_kernel(int n_sites, int n_bonds, const int32_t *bond_site, const int32_t *bond_dim,
                                      const int32_t *site_ptr, const int32_t *site_bonds, int32_t *bond_leg,
                                      int32_t *inc_slot, int64_t *tens_off)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    for (int b = 0; b < 2 * n_bonds; ++b) bond_leg[b] = -1;
    tens_off[0] = 0;
    for (int v = 0; v < n_sites; ++v) {
        int64_t n = 1;
        for (int i = site_ptr[v]; i < site_ptr[v + 1]; ++i) {
            const int b = site_bonds[i];
            bond_leg[2 * b + (bond_site[2 * b] == v ? 0 : 1)] = i - site_ptr[v];
            n *= bond_dim[b];
        }
        tens_off[v + 1] = tens_off[v] + n;
    }
    for (int v = 0; v < n_sites; ++v)
        for (int i = site_ptr[v]; i < site_ptr[v + 1]; ++i) {
            const int b = site_bonds[i];
            const int s0 = bond_site[2 * b], s1 = bond_site[2 * b + 1];
            if (s1 < 0) { inc_slot[i] = i; continue; }
            const int u = (s0 == v) ? s1 : s0, side = (s0 == v) ? 1 : 0;
            inc_slot[i] = site_ptr[u] + bond_leg[2 * b + side];
        }
}

__global__ void noalloc_copy_kernel(const double *msg, const int32_t *final_buf, int n_sets, int64_t per_set,
                                    double *out)
{
    const int64_t total = (int64_t)n_sets * per_set;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int set = (int)(i / per_set);
        out[i] = msg[((int64_t)final_buf[set] * n_sets) * per_set + i];
    }
}

// flag[0] = 1 when some tensor set did not converge (sweeps recorded as 0)
__global__ void noalloc_conv_kernel(const int32_t *iters, int n_sets, int32_t *flag)
{
    for (int i = threadIdx.x; i < n_sets; i += blockDim.x)
        if (iters[i] == 0) atomicExch(flag, 1);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace
}  // namespace pne

extern "C" pne_status pne_bp_messages_noalloc(const pne_network *net, double tol, int32_t max_iter, double *msg_out,
                                              int32_t *iters_out, double *residual_out, void *stream)
{
    using namespace pne;
    cudaStream_t s = (cudaStream_t)stream;
    if (!net || !msg_out || !net->bond_site || !net->bond_dim || !net->site_ptr || !net->site_bonds || !net->data ||
        !net->data_off || !net->data_on_device || net->n_sites < 1 || net->n_bonds < 0 || net->n_batch < 1) {
        set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: malformed network (device data required)");
        return PNE_EINVAL;
    }
    const int N = net->n_sites, M = net->n_bonds, B = net->n_batch;
    const int L = net->site_ptr[N];
    // host-side checks on the caller's arrays (nothing is allocated)
    int tabA = 1, tabC = 1;
    for (int b = 0; b < M; ++b) {
        const int s0 = net->bond_site[2 * b], s1 = net->bond_site[2 * b + 1];
        if (s0 < 0 || s0 >= N || s1 >= N || s1 < -1 || s0 == s1 || net->bond_dim[b] < 2 || net->bond_dim[b] > kMaxDim) {
            set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: invalid bond " + std::to_string(b));
            return PNE_EINVAL;
        }
    }
    if (net->site_ptr[0] != 0 || net->data_off[0] != 0) {
        set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: site_ptr[0] and data_off[0] must be 0");
        return PNE_EINVAL;
    }
    for (int v = 0; v < N; ++v)
        if (net->site_ptr[v + 1] < net->site_ptr[v] || net->site_ptr[v + 1] - net->site_ptr[v] > kMaxDeg) {
            set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: site degree must be in 0..6");
            return PNE_EINVAL;
        }
    // every bond listed exactly once at each of its sites
    for (int b = 0; b < M; ++b)
        for (int side = 0; side < 2; ++side) {
            const int x = net->bond_site[2 * b + side];
            if (x < 0) continue;
            int c = 0;
            for (int i = net->site_ptr[x]; i < net->site_ptr[x + 1]; ++i) c += (net->site_bonds[i] == b);
            if (c != 1) {
                set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: bond not listed once at each of its sites");
                return PNE_EINVAL;
            }
        }
    for (int v = 0; v < N; ++v) {
        const int a = net->site_ptr[v], e = net->site_ptr[v + 1], k = e - a, h = k / 2;
        if (k < 0 || k > kMaxDeg) { set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: site degree must be in 0..6"); return PNE_EINVAL; }
        int64_t size = 1;
        int A = 1, C = 1;
        for (int i = a; i < e; ++i) {
            const int b = net->site_bonds[i];
            if (b < 0 || b >= M || (i > a && net->site_bonds[i - 1] >= b) ||
                (net->bond_site[2 * b] != v && net->bond_site[2 * b + 1] != v)) {
                set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: bad leg list");
                return PNE_EINVAL;
            }
            size *= net->bond_dim[b];
            if (i - a < h) A *= net->bond_dim[b]; else C *= net->bond_dim[b];
        }
        if (size > 4096 || net->data_off[v + 1] - net->data_off[v] != size) {
            set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: data_off inconsistent or tensor above 4096 entries");
            return PNE_EINVAL;
        }
        tabA = tabA > A ? tabA : A;
        tabC = tabC > C ? tabC : C;
    }
    // scratch layout
    size_t off = 0;
    const size_t o_bs = off; off = align256(off + (size_t)2 * M * 4 + 4);
    const size_t o_bd = off; off = align256(off + (size_t)M * 4 + 4);
    const size_t o_sp = off; off = align256(off + (size_t)(N + 1) * 4);
    const size_t o_sb = off; off = align256(off + (size_t)L * 4 + 4);
    const size_t o_bl = off; off = align256(off + (size_t)2 * M * 4 + 4);
    const size_t o_is = off; off = align256(off + (size_t)L * 4 + 4);
    const size_t o_to = off; off = align256(off + (size_t)(N + 1) * 8);
    const size_t o_msg = off; off = align256(off + (size_t)2 * B * L * kMsgStride * 8);
    const size_t o_zero = off;                       // everything below starts at zero each call
    const size_t o_res = off; off = align256(off + (size_t)4 * B * 8);
    const size_t o_rout = off; off = align256(off + (size_t)B * 8);
    const size_t o_done = off; off = align256(off + (size_t)3 * B * 4);
    const size_t o_flags = off; off = align256(off + 16 + 8);
    if (off > PNE_NOALLOC_SCRATCH_BYTES) {
        set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: network needs " + std::to_string(off) +
                                       " bytes of scratch, above PNE_NOALLOC_SCRATCH_BYTES");
        return PNE_EINVAL;
    }
    const int per_warp = 2 * kMaxDeg * kMsgStride + 2 * tabA + 2 * tabC;
    const size_t smem = (size_t)per_warp * kBpWarps * sizeof(double);
    if (smem > 200 * 1024) { set_error(nullptr, PNE_EINVAL, "pne_bp_messages_noalloc: site tensor too large"); return PNE_EINVAL; }
    // device address of the array, once per device
    int dev = 0;
    PNE_CUDA_TRY(nullptr, cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) { set_error(nullptr, PNE_EINVAL, "device ordinal out of range"); return PNE_EINVAL; }
    if (!g_noalloc_addr[dev].load()) {
        void *ptr = nullptr;
        PNE_CUDA_TRY(nullptr, cudaGetSymbolAddress(&ptr, g_bp_noalloc_scratch));
        g_noalloc_addr[dev].store(ptr);
    }
    char *base = (char *)g_noalloc_addr[dev].load();
    int32_t *bs = (int32_t *)(base + o_bs), *bd = (int32_t *)(base + o_bd), *sp = (int32_t *)(base + o_sp);
    int32_t *sb = (int32_t *)(base + o_sb), *bl = (int32_t *)(base + o_bl), *is = (int32_t *)(base + o_is);
    int64_t *to = (int64_t *)(base + o_to);
    double *msg = (double *)(base + o_msg);
    unsigned long long *res = (unsigned long long *)(base + o_res);
    double *res_out = (double *)(base + o_rout);
    int32_t *done = (int32_t *)(base + o_done), *iters = done + B, *finalb = iters + B;
    int32_t *flags = (int32_t *)(base + o_flags);
    unsigned int *bar = (unsigned int *)(flags + 4);
    PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(bs, net->bond_site, (size_t)2 * M * 4, cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(bd, net->bond_dim, (size_t)M * 4, cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(sp, net->site_ptr, (size_t)(N + 1) * 4, cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(sb, net->site_bonds, (size_t)L * 4, cudaMemcpyHostToDevice, s));
    PNE_CUDA_TRY(nullptr, cudaMemsetAsync(base + o_zero, 0, off - o_zero, s));
    noalloc_tables_kernel<<<1, 1, 0, s>>>(N, M, bs, bd, sp, sb, bl, is, to);
    PNE_CUDA_TRY(nullptr, cudaGetLastError());
    int n_sm = 0;
    PNE_CUDA_TRY(nullptr, cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev));
    bp_init_kernel<<<grid_for((int64_t)B * L, 256, n_sm), 256, 0, s>>>(msg, sp, sb, bd, N, L, B);
    PNE_CUDA_TRY(nullptr, cudaGetLastError());
    BPParams prm;
    prm.n_sets = B; prm.n_sites = N; prm.n_legs = L;
    prm.site_ptr = sp; prm.site_bonds = sb; prm.bond_dim = bd; prm.inc_slot = is;
    prm.tens_off = to; prm.set_stride = net->data_off[N];
    prm.T = net->data; prm.msg = msg;
    prm.tol = (tol > 0) ? tol : 1e-13; prm.damping = 0.0; prm.max_iter = (max_iter > 0) ? max_iter : 10000;
    prm.res = res; prm.done_it = done; prm.iters_out = iters; prm.res_out = res_out;
    prm.final_buf = finalb; prm.flags = flags; prm.bar = bar;
    prm.smem_per_warp = per_warp; prm.tabA = tabA; prm.tabC = tabC;
    prm.n_colors = 0; prm.color_ptr = nullptr; prm.color_sites = nullptr;   // Jacobi sweeps, two buffers
    if (smem > 48 * 1024) {
        // only ever raised: a context may have granted this kernel more already
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, bp_persistent_kernel) != cudaSuccess || fa.maxDynamicSharedSizeBytes < (int)smem)
            PNE_CUDA_TRY(nullptr, grant_dynamic_smem((const void *)bp_persistent_kernel, smem));
    }
    int per_sm = 0;
    PNE_CUDA_TRY(nullptr, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bp_persistent_kernel, kBpWarps * 32, smem));
    if (per_sm < 1) { set_error(nullptr, PNE_EINVAL, "BP kernel does not fit"); return PNE_EINVAL; }
    const int64_t items = (int64_t)B * N;
    int64_t want = (items + kBpWarps - 1) / kBpWarps, cap = (int64_t)per_sm * n_sm;
    int nblocks = (int)(want < cap ? want : cap);
    if (nblocks < 1) nblocks = 1;
    void *args[] = {&prm};
    PNE_CUDA_TRY(nullptr, cudaLaunchCooperativeKernel((void *)bp_persistent_kernel, dim3(nblocks),
                                                       dim3(kBpWarps * 32), args, smem, s));
    const int64_t per_set = (int64_t)L * kMsgStride;
    noalloc_copy_kernel<<<grid_for((int64_t)B * per_set, 256, n_sm), 256, 0, s>>>(msg, finalb, B, per_set, msg_out);
    PNE_CUDA_TRY(nullptr, cudaGetLastError());
    // the convergence verdict of every set folded into one word on the device,
    // read back with the barrier and degeneracy flags in one copy on `s`
    noalloc_conv_kernel<<<1, 256, 0, s>>>(iters, B, flags + 2);
    PNE_CUDA_TRY(nullptr, cudaGetLastError());
    int32_t hflags[3] = {0, 0, 0};
    PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(hflags, flags, 12, cudaMemcpyDeviceToHost, s));
    if (iters_out) PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(iters_out, iters, (size_t)B * 4, cudaMemcpyDeviceToHost, s));
    if (residual_out) PNE_CUDA_TRY(nullptr, cudaMemcpyAsync(residual_out, res_out, (size_t)B * 8, cudaMemcpyDeviceToHost, s));
    PNE_CUDA_TRY(nullptr, cudaStreamSynchronize(s));
    if (hflags[0]) { set_error(nullptr, PNE_ETIMEOUT, "grid barrier timed out in BP"); return PNE_ETIMEOUT; }
    if (hflags[1]) { set_error(nullptr, PNE_EDEGENERATE, "zero BP message"); return PNE_EDEGENERATE; }
    if (hflags[2]) { set_error(nullptr, PNE_ENOCONV, "BP did not converge"); return PNE_ENOCONV; }
    return PNE_OK;
}
