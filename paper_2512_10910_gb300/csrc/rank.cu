// Rank-r projectors by weight passing (App. C) and the expansions built on
// them (Sec. V.A).
//
// Weight passing keeps a diagonal weight matrix S_i on every bond.  An update
// of bond i between tensors A and B (Eq. weight1-3) absorbs the weights of the
// other legs into A and B, takes the SVD of each (as a matrix between index i
// and the rest), then of S_A V_A^T S_i U_B S_B = U_C S_C V_C^T, and re-gauges
//     A <- A V_A S_A^{-1} U_C S_C^{(1-alpha)/2},
//     B <- S_C^{(1-alpha)/2} V_C^T S_B^{-1} U_B^T B,    S_i <- S_C^alpha,
// which leaves the network (with the weights inserted) unchanged.  Only the
// right singular vectors and values of the matricised tensors are needed: a
// Householder QR reduces each to a d x d triangle, whose SVD (and that of the
// d x d core) is taken by one-sided Jacobi rotations (Hestenes), in FP64.
// One thread block per tensor set runs the sweeps over the bonds in id order.
//
// The rank-r expansion restricts, per term, each bond's index to the P range
// [0, r) of the r largest weights, to the Q range [r, d), or leaves it whole,
// and contracts the weighted network exactly: a block per (term, tensor set)
// absorbs the sites one by one into a dense running tensor over the open
// frontier (FP64 multiply-adds).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "pne_internal.h"

struct pne_weights {
    pne_ctx *ctx = nullptr;
    std::shared_ptr<pne::GeomPair> geo;
    int n_sets = 1;
    pne::DevBuf T;           // [n_sets][stride] weighted network (sqrt(S) absorbed)
    pne::DevBuf S;           // [n_sets][n_bonds][16]
    std::vector<double> log_scale;
    std::vector<int32_t> sweeps;
    cudaStream_t last_stream = nullptr;
};

namespace pne {

// the geometry of a validated network through the context's cache (pne_api.cu)
pne_status geometry_for(pne_ctx *ctx, const pne_network *net, cudaStream_t s, std::shared_ptr<GeomPair> &out,
                        int max_dim, int64_t max_size);

namespace {

constexpr int kWpDim = 16;              // largest bond dimension of weight passing
constexpr int kWpThreads = 256;
constexpr int kWpWarps = kWpThreads / 32;

struct WPParams {
    int n_sets, n_sites, n_bonds;
    const int32_t *site_ptr, *site_bonds, *bond_dim, *bond_site, *bond_leg;
    const int64_t *tens_off;
    int64_t set_stride;
    double *T;                 // [n_sets][stride]: re-gauged in place, weighted at the end
    double *S;                 // [n_sets][n_bonds][kWpDim]
    double *scratch;           // [n_sets][scratch_per]
    int64_t scratch_per;
    double alpha, tol;
    int max_sweeps;
    double *log_scale;         // [n_sets]
    int32_t *sweeps;           // [n_sets] (0: not converged)
    int32_t *flags;            // [n_sets] 1: a zero singular value
};

__device__ double block_sum(double v, double *red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kWpWarps; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Tensor v of the set as a matrix [rest, d] (column = digit of leg l, rows =
// the other legs row-major), the weights of every other leg multiplied in,
// column-major into M (M[c * rest + row]).
__device__ void matricise(const WPParams &p, const double *Tset, const double *Sset, int v, int l, double *M,
                          int64_t &rest_out, int &d_out)
{
    const int l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
    int dims[kMaxDeg], bonds[kMaxDeg];
    for (int i = 0; i < k; ++i) { bonds[i] = p.site_bonds[l0 + i]; dims[i] = p.bond_dim[bonds[i]]; }
    const int64_t n = p.tens_off[v + 1] - p.tens_off[v];
    const int d = dims[l];
    const int64_t rest = n / d;
    const double *T = Tset + p.tens_off[v];
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        int64_t r = e, row = 0, mul = 1;
        int col = 0;
        double wgt = 1.0;
        for (int i = k - 1; i >= 0; --i) {
            const int dg = (int)(r % dims[i]);
            r /= dims[i];
            if (i == l) { col = dg; continue; }
            row += dg * mul;
            mul *= dims[i];
            wgt *= Sset[(int64_t)bonds[i] * kWpDim + dg];
        }
        M[(int64_t)col * rest + row] = T[e] * wgt;
    }
    rest_out = rest;
    d_out = d;
    __syncthreads();
}

// Householder QR of the column-major m x n matrix M (m >= n): the n x n
// upper triangle R goes to R (row-major, ldr = kWpDim).  A warp per column
// for the reflections' dot products.
__device__ void householder_r(double *M, int64_t m, int n, double *R, double *red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int j = 0; j < n; ++j) {
        double *x = M + (int64_t)j * m;
        double s = 0.0;
        for (int64_t i = j + threadIdx.x; i < m; i += blockDim.x) s += x[i] * x[i];
        s = block_sum(s, red);
        const double x0 = x[j];
        const double nrm = sqrt(s);
        const double alpha = (x0 >= 0.0) ? -nrm : nrm;
        const double vj = x0 - alpha;
        const double vn2 = s - x0 * x0 + vj * vj;
        __syncthreads();
        if (threadIdx.x == 0) x[j] = vj;
        __syncthreads();
        if (vn2 > 0.0) {
            const double beta = 2.0 / vn2;
            for (int c = j + 1 + warp; c < n; c += kWpWarps) {
                double *y = M + (int64_t)c * m;
                double dot = 0.0;
                for (int64_t i = j + lane; i < m; i += 32) dot += x[i] * y[i];
                for (int off = 16; off > 0; off >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, off);
                const double f = beta * dot;
                for (int64_t i = j + lane; i < m; i += 32) y[i] -= f * x[i];
            }
        }
        __syncthreads();
        if (threadIdx.x < n) {
            const int c = threadIdx.x;
            R[j * kWpDim + c] = (c < j) ? 0.0 : (c == j ? alpha : M[(int64_t)c * m + j]);
        }
        __syncthreads();
    }
}

// One-sided Jacobi SVD of the n x n row-major W (ld kWpDim): on return W's
// columns are U * sigma, V (row-major, ld kWpDim) the right singular vectors
// and sig the singular values, sorted descending (columns permuted alike).
// One warp, a lane per row.
__device__ void jacobi_svd(double *W, double *V, double *sig, int n)
{
    const int lane = threadIdx.x & 31;
    for (int c = 0; c < n; ++c)
        if (lane < n) V[lane * kWpDim + c] = (lane == c) ? 1.0 : 0.0;
    __syncwarp();
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                const double wp = lane < n ? W[lane * kWpDim + p] : 0.0;
                const double wq = lane < n ? W[lane * kWpDim + q] : 0.0;
                double a = wp * wp, b = wq * wq, g = wp * wq;
                for (int off = 16; off > 0; off >>= 1) {
                    a += __shfl_xor_sync(0xffffffffu, a, off);
                    b += __shfl_xor_sync(0xffffffffu, b, off);
                    g += __shfl_xor_sync(0xffffffffu, g, off);
                }
                if (fabs(g) <= 1e-15 * sqrt(a * b) || g == 0.0) continue;
                rotated = 1;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                if (lane < n) {
                    W[lane * kWpDim + p] = cs * wp - sn * wq;
                    W[lane * kWpDim + q] = sn * wp + cs * wq;
                    const double vp = V[lane * kWpDim + p], vq = V[lane * kWpDim + q];
                    V[lane * kWpDim + p] = cs * vp - sn * vq;
                    V[lane * kWpDim + q] = sn * vp + cs * vq;
                }
                __syncwarp();
            }
        if (!rotated) break;
    }
    for (int c = 0; c < n; ++c) {
        const double w = lane < n ? W[lane * kWpDim + c] : 0.0;
        double s2 = w * w;
        for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        if (lane == 0) sig[c] = sqrt(s2);
    }
    __syncwarp();
    // selection sort by singular value, descending (columns of W and V move along)
    for (int i = 0; i < n; ++i) {
        int best = i;
        for (int c = i + 1; c < n; ++c) if (sig[c] > sig[best]) best = c;
        if (best != i) {
            if (lane < n) {
                double t = W[lane * kWpDim + i]; W[lane * kWpDim + i] = W[lane * kWpDim + best]; W[lane * kWpDim + best] = t;
                t = V[lane * kWpDim + i]; V[lane * kWpDim + i] = V[lane * kWpDim + best]; V[lane * kWpDim + best] = t;
            }
            __syncwarp();
            if (lane == 0) { const double t = sig[i]; sig[i] = sig[best]; sig[best] = t; }
        }
        __syncwarp();
    }
}

// T_v <- T_v with leg l multiplied by the d x d matrix X: new[.., c, ..] =
// sum_a old[.., a, ..] X[a][c] when right == 0, or sum_a X[c][a] old[.., a, ..]
// when right == 1.  `tmp` holds a copy of the tensor.
__device__ void apply_leg(const WPParams &p, double *Tset, int v, int l, const double *X, int right, double *tmp)
{
    const int l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
    int dims[kMaxDeg];
    for (int i = 0; i < k; ++i) dims[i] = p.bond_dim[p.site_bonds[l0 + i]];
    int64_t post = 1;
    for (int i = l + 1; i < k; ++i) post *= dims[i];
    const int d = dims[l];
    const int64_t n = p.tens_off[v + 1] - p.tens_off[v];
    double *T = Tset + p.tens_off[v];
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) tmp[e] = T[e];
    __syncthreads();
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
        const int64_t lo = e % post, hi = e / post / d;
        const int c = (int)((e / post) % d);
        double acc = 0.0;
        for (int a = 0; a < d; ++a) {
            const double m = right ? X[c * kWpDim + a] : X[a * kWpDim + c];
            acc = fma(tmp[(hi * d + a) * post + lo], m, acc);
        }
        T[e] = acc;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kWpThreads) weight_passing_kernel(WPParams p)
{
    __shared__ double red[kWpWarps];
    __shared__ double RA[kWpDim * kWpDim], VA[kWpDim * kWpDim], RB[kWpDim * kWpDim], VB[kWpDim * kWpDim];
    __shared__ double MC[kWpDim * kWpDim], VC[kWpDim * kWpDim], X[kWpDim * kWpDim];
    __shared__ double sA[kWpDim], sB[kWpDim], sC[kWpDim];
    __shared__ double change_sh, scale_sh;
    __shared__ int bad_sh;
    const int set = blockIdx.x;
    if (set >= p.n_sets) return;
    double *Tset = p.T + (int64_t)set * p.set_stride;
    double *Sset = p.S + (int64_t)set * p.n_bonds * kWpDim;
    double *buf = p.scratch + (int64_t)set * p.scratch_per;
    for (int64_t i = threadIdx.x; i < (int64_t)p.n_bonds * kWpDim; i += blockDim.x)
        Sset[i] = ((int)(i % kWpDim) < p.bond_dim[i / kWpDim]) ? 1.0 : 0.0;
    if (threadIdx.x == 0) { scale_sh = 0.0; bad_sh = 0; }
    __syncthreads();
    int done = 0;
    for (int sweep = 1; sweep <= p.max_sweeps && !done; ++sweep) {
        if (threadIdx.x == 0) change_sh = 0.0;
        __syncthreads();
        for (int b = 0; b < p.n_bonds; ++b) {
            const int u = p.bond_site[2 * b], v = p.bond_site[2 * b + 1];
            const int lu = p.bond_leg[2 * b], lv = p.bond_leg[2 * b + 1];
            int64_t mA, mB;
            int d, d2;
            // A' and B' (other legs' weights absorbed), reduced to triangles
            matricise(p, Tset, Sset, u, lu, buf, mA, d);
            householder_r(buf, mA, d, RA, red);
            matricise(p, Tset, Sset, v, lv, buf, mB, d2);
            householder_r(buf, mB, d, RB, red);
            if (threadIdx.x < 32) {
                jacobi_svd(RA, VA, sA, d);      // right vectors V_A, values S_A
                jacobi_svd(RB, VB, sB, d);      // B'^T: right vectors U_B, values S_B
            }
            __syncthreads();
            if (threadIdx.x == 0)
                for (int a = 0; a < d; ++a) if (!(sA[a] > 1e-300) || !(sB[a] > 1e-300)) bad_sh = 1;
            __syncthreads();
            if (bad_sh) break;
            // core M = S_A V_A^T S_i U_B S_B and its SVD
            const double *Si = Sset + (int64_t)b * kWpDim;
            for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
                const int a = e / d, c = e % d;
                double acc = 0.0;
                for (int x = 0; x < d; ++x) acc = fma(VA[x * kWpDim + a] * Si[x], VB[x * kWpDim + c], acc);
                MC[a * kWpDim + c] = sA[a] * acc * sB[c];
            }
            __syncthreads();
            if (threadIdx.x < 32) jacobi_svd(MC, VC, sC, d);     // MC -> U_C S_C, VC = V_C
            __syncthreads();
            if (threadIdx.x == 0) {
                double mx = 0.0;
                for (int a = 0; a < d; ++a) mx = fmax(mx, pow(sC[a], p.alpha));
                if (!(sC[d - 1] > 1e-300)) bad_sh = 1;
                scale_sh += log(mx);
                double ch = change_sh;
                for (int a = 0; a < d; ++a) {
                    const double nw = pow(sC[a], p.alpha) / mx;
                    ch = fmax(ch, fabs(nw - Sset[(int64_t)b * kWpDim + a]));
                    Sset[(int64_t)b * kWpDim + a] = nw;
                }
                change_sh = ch;
            }
            __syncthreads();
            if (bad_sh) break;
            // left = V_A S_A^{-1} U_C S_C^{(1-alpha)/2} on A's leg
            for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
                const int a = e / d, c = e % d;
                double acc = 0.0;
                for (int x = 0; x < d; ++x) acc = fma(VA[a * kWpDim + x] / sA[x], MC[x * kWpDim + c] / sC[c], acc);
                X[a * kWpDim + c] = acc * pow(sC[c], 0.5 * (1.0 - p.alpha));
            }
            __syncthreads();
            apply_leg(p, Tset, u, lu, X, 0, buf);
            // right = S_C^{(1-alpha)/2} V_C^T S_B^{-1} U_B^T on B's leg
            for (int e = threadIdx.x; e < d * d; e += blockDim.x) {
                const int c = e / d, a = e % d;
                double acc = 0.0;
                for (int x = 0; x < d; ++x) acc = fma(VC[x * kWpDim + c] / sB[x], VB[a * kWpDim + x], acc);
                X[c * kWpDim + a] = pow(sC[c], 0.5 * (1.0 - p.alpha)) * acc;
            }
            __syncthreads();
            apply_leg(p, Tset, v, lv, X, 1, buf);
        }
        __syncthreads();
        if (bad_sh) break;
        if (change_sh < p.tol) {
            done = 1;
            if (threadIdx.x == 0) p.sweeps[set] = sweep;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (!done) p.sweeps[set] = 0;
        p.flags[set] = bad_sh;
        p.log_scale[set] = scale_sh;
    }
    // the weighted network: sqrt(S) into both ends of every bond
    for (int v = 0; v < p.n_sites; ++v) {
        const int l0 = p.site_ptr[v], k = p.site_ptr[v + 1] - l0;
        int dims[kMaxDeg], bonds[kMaxDeg];
        for (int i = 0; i < k; ++i) { bonds[i] = p.site_bonds[l0 + i]; dims[i] = p.bond_dim[bonds[i]]; }
        const int64_t n = p.tens_off[v + 1] - p.tens_off[v];
        double *T = Tset + p.tens_off[v];
        for (int64_t e = threadIdx.x; e < n; e += blockDim.x) {
            int64_t r = e;
            double w = 1.0;
            for (int i = k - 1; i >= 0; --i) {
                const int dg = (int)(r % dims[i]);
                r /= dims[i];
                w *= sqrt(Sset[(int64_t)bonds[i] * kWpDim + dg]);
            }
            T[e] *= w;
        }
    }
}

// ---------------------------------------------------------------- dense terms
constexpr int kDtThreads = 256;
constexpr int64_t kDtMaxFront = 1 << 18;      // entries of a running tensor
constexpr int kDtMaxLegs = 20;                // bonds of a frontier
constexpr int kDtMaxBonds = 1024;             // bonds of a network

// One step of the site-by-site contraction: the site absorbed, the frontier
// before (bond ids, in order) and after, and for each leg of the site its
// position in the old frontier (closing) or the new one (opening).
struct DtStep {
    int site, k, nf0, nf1;
    int f0[kDtMaxLegs];
    int f1[kDtMaxLegs];
    int leg_bond[kMaxDeg];
    int leg_old[kMaxDeg];       // position in f0, or -1
    int leg_new[kMaxDeg];       // position in f1, or -1
    int keep_new[kDtMaxLegs];   // for each position of f1: position in f0 (kept) or -1 (a new leg)
};

struct DtParams {
    const DtStep *steps;
    int n_steps, n_bonds, n_terms, n_sets;
    const int8_t *kind;          // [n_terms][n_bonds]: 0 whole, 1 P range, 2 Q range
    const int32_t *bond_dim;
    int rank;
    const double *T;             // [n_sets][stride] weighted network
    const int64_t *tens_off;
    int64_t set_stride;
    double *scratch;             // [grid][2][kDtMaxFront]
    double *value;               // [n_sets][n_terms]
};

__global__ void __launch_bounds__(kDtThreads) dense_term_kernel(DtParams p)
{
    __shared__ int lo[kDtMaxBonds], len[kDtMaxBonds];
    double *X = p.scratch + (int64_t)blockIdx.x * 2 * kDtMaxFront;
    double *Y = X + kDtMaxFront;
    const int64_t items = (int64_t)p.n_terms * p.n_sets;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int term = (int)(item % p.n_terms), set = (int)(item / p.n_terms);
        for (int b = threadIdx.x; b < p.n_bonds; b += blockDim.x) {
            const int kd = p.kind[(int64_t)term * p.n_bonds + b], d = p.bond_dim[b];
            lo[b] = (kd == 2) ? p.rank : 0;
            len[b] = (kd == 0) ? d : (kd == 1 ? p.rank : d - p.rank);
        }
        if (threadIdx.x == 0) X[0] = 1.0;
        __syncthreads();
        const double *Tset = p.T + (int64_t)set * p.set_stride;
        for (int s = 0; s < p.n_steps; ++s) {
            const DtStep &st = p.steps[s];
            // sizes and row-major strides of the old and new frontiers
            int64_t n1 = 1;
            for (int i = 0; i < st.nf1; ++i) n1 *= len[st.f1[i]];
            int64_t str0[kDtMaxLegs];
            {
                int64_t m = 1;
                for (int i = st.nf0 - 1; i >= 0; --i) { str0[i] = m; m *= len[st.f0[i]]; }
            }
            int cl_len[kMaxDeg], cl_pos[kMaxDeg], nc = 0;
            int64_t ncomb = 1;
            for (int l = 0; l < st.k; ++l)
                if (st.leg_old[l] >= 0) { cl_pos[nc] = l; cl_len[nc] = len[st.leg_bond[l]]; ncomb *= cl_len[nc]; ++nc; }
            int dims[kMaxDeg];
            for (int l = 0; l < st.k; ++l) dims[l] = p.bond_dim[st.leg_bond[l]];
            const double *Tv = Tset + p.tens_off[st.site];
            for (int64_t o = threadIdx.x; o < n1; o += blockDim.x) {
                // digits of the new frontier (last fastest)
                int dg1[kDtMaxLegs];
                int64_t r = o;
                for (int i = st.nf1 - 1; i >= 0; --i) { const int L = len[st.f1[i]]; dg1[i] = (int)(r % L); r /= L; }
                int64_t xbase = 0;
                for (int i = 0; i < st.nf1; ++i)
                    if (st.keep_new[i] >= 0) xbase += dg1[i] * str0[st.keep_new[i]];
                int tdg[kMaxDeg];
                for (int l = 0; l < st.k; ++l)
                    tdg[l] = (st.leg_new[l] >= 0) ? lo[st.leg_bond[l]] + dg1[st.leg_new[l]] : 0;
                double acc = 0.0;
                for (int64_t c = 0; c < ncomb; ++c) {
                    int64_t rc = c, xo = xbase;
                    for (int j = nc - 1; j >= 0; --j) {
                        const int l = cl_pos[j];
                        const int dg = (int)(rc % cl_len[j]);
                        rc /= cl_len[j];
                        xo += dg * str0[st.leg_old[l]];
                        tdg[l] = lo[st.leg_bond[l]] + dg;
                    }
                    int64_t to = 0;
                    for (int l = 0; l < st.k; ++l) to = to * dims[l] + tdg[l];
                    acc = fma(X[xo], Tv[to], acc);
                }
                Y[o] = acc;
            }
            __syncthreads();
            double *t = X; X = Y; Y = t;
        }
        if (threadIdx.x == 0) p.value[(int64_t)set * p.n_terms + term] = X[0];
        __syncthreads();
        // X, Y alternate per step: restore the block's buffer order
        X = p.scratch + (int64_t)blockIdx.x * 2 * kDtMaxFront;
        Y = X + kDtMaxFront;
    }
}

// One term's tensors with every bond's index restricted to [lo_b, lo_b + len_b):
// block per (site, set), row-major over the site's legs in ascending bond id.
__global__ void restrict_kernel(const double *__restrict__ T, int64_t set_stride, const int64_t *tens_off,
                                const int32_t *site_ptr, const int32_t *site_bonds, const int32_t *bond_dim,
                                const int32_t *lo, const int32_t *len, const int64_t *new_off, int64_t new_stride,
                                double *out)
{
    const int v = blockIdx.x, set = blockIdx.y;
    const int p0 = site_ptr[v], p1 = site_ptr[v + 1];
    const int64_t n_out = new_off[v + 1] - new_off[v];
    const double *src = T + set * set_stride + tens_off[v];
    double *dst = out + set * new_stride + new_off[v];
    for (int64_t q = threadIdx.x; q < n_out; q += blockDim.x) {
        int64_t r = q, off = 0, stride = 1;
        for (int i = p1 - 1; i >= p0; --i) {
            const int b = site_bonds[i];
            const int64_t digit = r % len[b];
            r /= len[b];
            off += (lo[b] + digit) * stride;
            stride *= bond_dim[b];
        }
        dst[q] = src[off];
    }
}

struct RankTerms {
    std::vector<int8_t> kind;       // [n_terms][n_bonds]: 0 whole, 1 P range, 2 Q range
    std::vector<int> order, sign;
    int M = 0;
};

pne_status rank_terms(pne_ctx *ctx, const Geometry &g, int32_t rank, int32_t form, int32_t n_partitions,
                      const int32_t *partition_ptr, const int32_t *partition_bonds, RankTerms &t)
{
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    const int M = n_partitions, NB = g.n_bonds;
    if (M < 1 || M > 20) return bad("1..20 partitions");
    if (form != 0 && form != 1) return bad("form is 0 (linear) or 1 (combinatorial)");
    if (partition_ptr[0] != 0) return bad("partition_ptr[0] must be 0");
    std::vector<std::vector<int>> parts(M);
    for (int p = 0; p < M; ++p) {
        if (partition_ptr[p + 1] <= partition_ptr[p]) return bad("every partition needs at least one bond");
        for (int i = partition_ptr[p]; i < partition_ptr[p + 1]; ++i) {
            const int b = partition_bonds[i];
            if (b < 0 || b >= NB) return bad("partition bond out of range");
            if (rank < 1 || rank >= g.bond_dim[b]) return bad("rank must be in 1 .. d - 1 on every partitioned bond");
            parts[p].push_back(b);
        }
        if (form == 0 && parts[p].size() != 1) return bad("the linear form takes single-index partitions");
    }
    if (form == 0)
        for (int p = 0; p < M; ++p)
            for (int q = p + 1; q < M; ++q)
                if (parts[p][0] == parts[q][0]) return bad("the linear form takes distinct bonds");
    t.M = M;
    t.kind.clear();
    t.order.clear();
    t.sign.clear();
    if (form == 0) {
        for (int k = 0; k < M; ++k) {
            std::vector<int8_t> row(NB, 0);
            for (int p = 0; p < k; ++p) row[parts[p][0]] = 2;
            row[parts[k][0]] = 1;
            t.kind.insert(t.kind.end(), row.begin(), row.end());
            t.order.push_back(k);
            t.sign.push_back(1);
        }
    } else {
        for (uint32_t x = 1; x < (1u << M); ++x) {
            std::vector<int8_t> row(NB, 0);
            int k = 0;
            for (int p = 0; p < M; ++p)
                if (x >> p & 1) { ++k; for (int b : parts[p]) row[b] = 1; }
            t.kind.insert(t.kind.end(), row.begin(), row.end());
            t.order.push_back(k);
            t.sign.push_back((k % 2 == 1) ? 1 : -1);
        }
    }
    return PNE_OK;
}

// per set: c[k], abs_c[k], the signed Neumaier sum of the term values (in the
// weighted network's scale), log_abs with the weights' log scale, and the
// a-priori bound: FP64 rounding of nops operations per term plus, for a
// reduced-precision contraction, bound_abs[set][term] = the contraction's
// relative bound x |value| (relative to each term's absolute contraction,
// which equals |value| for a term of non-negative tensors)
void rank_results(const pne_weights *w, int form, const RankTerms &t, const std::vector<double> &vals,
                  const std::vector<double> &bound_abs, int nops, pne_result *out)
{
    const int n_terms = (int)t.order.size();
    for (int set = 0; set < w->n_sets; ++set) {
        pne_result &r = out[set];
        std::memset(&r, 0, sizeof r);
        const int K = form == 0 ? t.M - 1 : t.M;
        r.n_orders = K + 1;
        double sum = 0.0, comp = 0.0, asum = 0.0, rb = 0.0;
        for (int q = 0; q < n_terms; ++q) {
            const double v = vals[(size_t)set * n_terms + q];
            r.c[t.order[q]] += v;
            r.abs_c[t.order[q]] += std::fabs(v);
        }
        for (int q = 0; q < n_terms; ++q) {            // Neumaier over the terms, in term order
            const double x = t.sign[q] * vals[(size_t)set * n_terms + q], tt = sum + x;
            comp += (std::fabs(sum) >= std::fabs(x)) ? (sum - tt) + x : (x - tt) + sum;
            sum = tt;
            asum += std::fabs(x);
            if (!bound_abs.empty()) rb += bound_abs[(size_t)set * n_terms + q];
        }
        sum += comp;
        const double ls = w->log_scale[set];
        r.log_abs_zref = ls;
        r.sign_zref = 1;
        r.sign = sum < 0 ? -1 : 1;
        r.log_abs = (sum != 0.0) ? ls + std::log(std::fabs(sum)) : -std::numeric_limits<double>::infinity();
        r.value = (sum == 0.0) ? 0.0 : (r.log_abs > 709.7 ? r.sign * std::numeric_limits<double>::infinity()
                                                           : r.sign * std::exp(r.log_abs));
        r.log_series = std::numeric_limits<double>::quiet_NaN();
        const double u = 0x1p-53;
        r.err_bound = (sum != 0.0) ? ((nops * u / (1 - nops * u)) * asum + rb) / std::fabs(sum)
                                   : std::numeric_limits<double>::infinity();
        r.n_terms = (uint64_t)n_terms;
        r.bp_iters = w->sweeps[set];
    }
}

// Every term network (bond kinds per term: 0 whole, 1 P range [0, rank), 2 Q
// range [rank, d)) contracted as a grid: the restricted tensors gathered per
// term, then the row-by-row GEMMs.  vals / bound_abs [set][term].
pne_status grid_term_values(pne_ctx *ctx, const pne_weights *w, const std::vector<int8_t> &kind, int n_terms,
                            int32_t rank, int32_t lx, int32_t ly, pne_dtype dtype, cudaStream_t s,
                            std::vector<double> &vals, std::vector<double> &bound_abs)
{
    const Geometry &g = w->geo->full;
    const int NB = g.n_bonds, ns = w->n_sets;
    vals.assign((size_t)ns * n_terms, 0.0);
    bound_abs.assign((size_t)ns * n_terms, 0.0);
    std::vector<int32_t> lo((size_t)NB), len((size_t)NB);
    std::vector<int64_t> off((size_t)g.n_sites + 1);
    DevBuf dlo, dlen, doff, ddata;
    auto cleanup = [&]() { dev_free(ctx, dlo, s); dev_free(ctx, dlen, s); dev_free(ctx, doff, s); dev_free(ctx, ddata, s); };
    pne_status st;
    if ((st = dev_alloc(ctx, dlo, (size_t)NB * 4, s)) || (st = dev_alloc(ctx, dlen, (size_t)NB * 4, s)) ||
        (st = dev_alloc(ctx, doff, off.size() * 8, s)) ||
        (st = dev_alloc(ctx, ddata, (size_t)ns * g.tens_off[g.n_sites] * 8, s))) {
        cleanup();
        return st;
    }
    for (int q = 0; q < n_terms; ++q) {
        for (int b = 0; b < NB; ++b) {
            const int kd = kind[(size_t)q * NB + b], d = g.bond_dim[b];
            lo[(size_t)b] = kd == 2 ? rank : 0;
            len[(size_t)b] = kd == 0 ? d : (kd == 1 ? rank : d - rank);
        }
        off[0] = 0;
        for (int v = 0; v < g.n_sites; ++v) {
            int64_t sz = 1;
            for (int i = g.site_ptr[v]; i < g.site_ptr[v + 1]; ++i) sz *= len[(size_t)g.site_bonds[i]];
            off[(size_t)v + 1] = off[(size_t)v] + sz;
        }
        GridPlan plan;
        if ((st = grid_plan(ctx, lx, ly, NB, g.bond_site.data(), len.data(), g.site_ptr.data(), g.site_bonds.data(),
                            off.data(), dtype, ns, plan)) ||
            (st = upload(ctx, dlo.ptr, lo.data(), (size_t)NB * 4, s)) ||
            (st = upload(ctx, dlen.ptr, len.data(), (size_t)NB * 4, s)) ||
            (st = upload(ctx, doff.ptr, off.data(), off.size() * 8, s))) {
            cleanup();
            return st;
        }
        {
            ProfScope ps(ctx, s, "rank_restrict");
            restrict_kernel<<<dim3(g.n_sites, ns), 256, 0, s>>>((const double *)w->T.ptr, g.tens_off[g.n_sites],
                                                                g.d_tens_off, g.d_site_ptr, g.d_site_bonds,
                                                                g.d_bond_dim, (const int32_t *)dlo.ptr,
                                                                (const int32_t *)dlen.ptr, (const int64_t *)doff.ptr,
                                                                off[(size_t)g.n_sites], (double *)ddata.ptr);
        }
        if (cudaGetLastError() != cudaSuccess) {
            cleanup();
            set_error(ctx, PNE_ECUDA, "restrict_kernel launch failed");
            return PNE_ECUDA;
        }
        std::vector<double> h;
        double bound = 0.0;
        if ((st = grid_run(ctx, plan, (const double *)ddata.ptr, off[(size_t)g.n_sites], ns, dtype, s, h, bound))) {
            cleanup();
            return st;
        }
        for (int set = 0; set < ns; ++set) {
            const double v = std::ldexp(h[2 * (size_t)set], (int)h[2 * (size_t)set + 1]);
            vals[(size_t)set * n_terms + q] = v;
            bound_abs[(size_t)set * n_terms + q] = dtype == PNE_F64 ? 0.0 : bound * std::fabs(v);
        }
    }
    cleanup();
    return PNE_OK;
}

}  // namespace
}  // namespace pne

// ======================================================================= host
using namespace pne;

namespace {

// Site order of the dense contraction: from site 0, repeatedly the site whose
// absorption leaves the smallest frontier (whole dimensions), ties by id; the
// steps record the frontiers before and after and where each leg goes.
pne_status dense_plan(pne_ctx *ctx, const Geometry &g, std::vector<DtStep> &steps, int64_t &max_front)
{
    const int N = g.n_sites;
    std::vector<char> in(N, 0);
    std::vector<int> front;                 // frontier bonds, in order
    max_front = 1;
    for (int s = 0; s < N; ++s) {
        int best = -1;
        double best_size = 0.0;
        for (int v = 0; v < N; ++v) {
            if (in[v]) continue;
            double size = 1.0;
            for (int b : front) {
                const bool closes = g.bond_site[2 * b] == v || g.bond_site[2 * b + 1] == v;
                if (!closes) size *= g.bond_dim[b];
            }
            for (int i = g.site_ptr[v]; i < g.site_ptr[v + 1]; ++i) {
                const int b = g.site_bonds[i];
                const int o = g.bond_site[2 * b] == v ? g.bond_site[2 * b + 1] : g.bond_site[2 * b];
                if (!in[o]) size *= g.bond_dim[b];
            }
            // prefer a site that touches the frontier (keeps components together)
            bool touches = front.empty();
            for (int b : front)
                if (g.bond_site[2 * b] == v || g.bond_site[2 * b + 1] == v) touches = true;
            const double key = touches ? size : size * 1e30;
            if (best < 0 || key < best_size) { best = v; best_size = key; }
        }
        const int v = best;
        DtStep st;
        std::memset(&st, 0, sizeof st);
        st.site = v;
        st.k = g.site_ptr[v + 1] - g.site_ptr[v];
        st.nf0 = (int)front.size();
        if (st.nf0 > kDtMaxLegs) { set_error(ctx, PNE_EINVAL, "frontier of the dense contraction too wide"); return PNE_EINVAL; }
        for (int i = 0; i < st.nf0; ++i) st.f0[i] = front[i];
        std::vector<int> nf;
        std::vector<int> keep;
        for (int i = 0; i < st.nf0; ++i) {
            const int b = front[i];
            if (g.bond_site[2 * b] == v || g.bond_site[2 * b + 1] == v) continue;
            nf.push_back(b);
            keep.push_back(i);
        }
        for (int l = 0; l < st.k; ++l) {
            const int b = g.site_bonds[g.site_ptr[v] + l];
            st.leg_bond[l] = b;
            st.leg_old[l] = -1;
            st.leg_new[l] = -1;
            for (int i = 0; i < st.nf0; ++i) if (front[i] == b) st.leg_old[l] = i;
            if (st.leg_old[l] < 0) {
                const int o = g.bond_site[2 * b] == v ? g.bond_site[2 * b + 1] : g.bond_site[2 * b];
                if (!in[o]) { st.leg_new[l] = (int)nf.size(); nf.push_back(b); keep.push_back(-1); }
            }
        }
        st.nf1 = (int)nf.size();
        if (st.nf1 > kDtMaxLegs) { set_error(ctx, PNE_EINVAL, "frontier of the dense contraction too wide"); return PNE_EINVAL; }
        int64_t size = 1;
        for (int i = 0; i < st.nf1; ++i) { st.f1[i] = nf[i]; st.keep_new[i] = keep[i]; size *= g.bond_dim[nf[i]]; }
        max_front = std::max(max_front, size);
        if (size > kDtMaxFront) {
            set_error(ctx, PNE_EINVAL, "an intermediate tensor of the dense contraction exceeds 2^18 entries");
            return PNE_EINVAL;
        }
        in[v] = 1;
        front = nf;
        steps.push_back(st);
    }
    return PNE_OK;
}

}  // namespace

extern "C" {

pne_status pne_weight_passing(pne_ctx *ctx, const pne_network *net, double alpha, double tol, int32_t max_sweeps,
                              void *stream, pne_weights **out)
{
    HostScope hs__(ctx, "weight_passing");
    if (!ctx || !net || !out) return PNE_EINVAL;
    *out = nullptr;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    if (!(alpha > 0.0 && alpha <= 1.0) || !(tol > 0.0) || max_sweeps < 1) return bad("alpha in (0, 1], tol > 0, max_sweeps > 0");
    cudaStream_t s = (cudaStream_t)stream;
    auto w = new pne_weights();
    w->ctx = ctx;
    // bond dimensions up to 16 and site tensors up to 2^20 entries here
    pne_status st = geometry_for(ctx, net, s, w->geo, kWpDim, (int64_t)1 << 20);
    if (st) { delete w; return st; }
    const Geometry &g = w->geo->full;
    if (!w->geo->open_bonds.empty()) { delete w; return bad("weight passing takes closed networks"); }
    for (int b = 0; b < g.n_bonds; ++b) {
        if (g.bond_dim[b] > kWpDim) { delete w; return bad("weight passing needs bond dimensions <= 16"); }
        for (int side = 0; side < 2; ++side) {
            const int v = g.bond_site[2 * b + side];
            const int64_t n = g.tens_off[v + 1] - g.tens_off[v];
            if (n / g.bond_dim[b] < g.bond_dim[b]) {
                delete w;
                return bad("a bond dimension exceeds the product of the other dimensions of its tensor");
            }
        }
    }
    const int B = net->n_batch;
    w->n_sets = B;
    const int64_t stride = g.tens_off[g.n_sites];
    int64_t tmax = 1;
    for (int v = 0; v < g.n_sites; ++v) tmax = std::max<int64_t>(tmax, g.tens_off[v + 1] - g.tens_off[v]);
    DevBuf scratch, rec;
    if ((st = dev_alloc(ctx, w->T, (size_t)B * stride * 8, s)) ||
        (st = dev_alloc(ctx, w->S, (size_t)B * std::max(g.n_bonds, 1) * kWpDim * 8, s)) ||
        (st = dev_alloc(ctx, scratch, (size_t)B * tmax * 8, s)) || (st = dev_alloc(ctx, rec, (size_t)B * 16, s))) {
        dev_free(ctx, scratch, s); dev_free(ctx, rec, s); pne_weights_destroy(w);
        return st;
    }
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(w->T.ptr, net->data, (size_t)B * stride * 8,
                                      net->data_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    WPParams p;
    p.n_sets = B; p.n_sites = g.n_sites; p.n_bonds = g.n_bonds;
    p.site_ptr = g.d_site_ptr; p.site_bonds = g.d_site_bonds; p.bond_dim = g.d_bond_dim; p.bond_site = g.d_bond_site;
    p.bond_leg = g.d_bond_leg; p.tens_off = g.d_tens_off; p.set_stride = stride;
    p.T = (double *)w->T.ptr; p.S = (double *)w->S.ptr;
    p.scratch = (double *)scratch.ptr; p.scratch_per = tmax;
    p.alpha = alpha; p.tol = tol; p.max_sweeps = max_sweeps;
    p.log_scale = (double *)rec.ptr;
    p.sweeps = (int32_t *)((char *)rec.ptr + (size_t)B * 8);
    p.flags = p.sweeps + B;
    {
        ProfScope ps(ctx, s, "weight_passing");
        weight_passing_kernel<<<B, kWpThreads, 0, s>>>(p);
    }
    PNE_LAUNCH_CHECK(ctx);
    std::vector<char> h((size_t)B * 16);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), rec.ptr, h.size(), cudaMemcpyDeviceToHost, s));
    dev_free(ctx, scratch, s);
    dev_free(ctx, rec, s);
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    w->log_scale.assign((const double *)h.data(), (const double *)h.data() + B);
    const int32_t *sw = (const int32_t *)(h.data() + (size_t)B * 8);
    w->sweeps.assign(sw, sw + B);
    w->last_stream = s;
    *out = w;
    for (int b = 0; b < B; ++b)
        if (sw[B + b]) { set_error(ctx, PNE_EDEGENERATE, "a zero singular value in weight passing"); return PNE_EDEGENERATE; }
    for (int b = 0; b < B; ++b)
        if (sw[b] == 0) { set_error(ctx, PNE_ENOCONV, "weight passing did not converge for a tensor set"); return PNE_ENOCONV; }
    return PNE_OK;
}

pne_status pne_weights_read(pne_ctx *ctx, const pne_weights *w, void *stream, double *weights, int32_t *sweeps,
                            double *log_scale)
{
    if (!ctx || !w) return PNE_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (weights) {
        const size_t n = (size_t)w->n_sets * std::max(w->geo->full.n_bonds, 1) * kWpDim;
        PNE_CUDA_TRY(ctx, cudaMemcpyAsync(weights, w->S.ptr, n * 8, cudaMemcpyDeviceToHost, s));
        PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    }
    if (sweeps) std::copy(w->sweeps.begin(), w->sweeps.end(), sweeps);
    if (log_scale) std::copy(w->log_scale.begin(), w->log_scale.end(), log_scale);
    return PNE_OK;
}

void pne_weights_destroy(pne_weights *w)
{
    if (!w) return;
    dev_free(w->ctx, w->T, w->last_stream);
    dev_free(w->ctx, w->S, w->last_stream);
    if (w->geo) w->geo->uses.note(w->ctx, w->last_stream);
    delete w;
}

pne_status pne_rank_r_expand(pne_ctx *ctx, const pne_weights *w, int32_t rank, int32_t form, int32_t n_partitions,
                             const int32_t *partition_ptr, const int32_t *partition_bonds, void *stream,
                             pne_result *out)
{
    HostScope hs__(ctx, "rank_r_expand");
    if (!ctx || !w || !out || !partition_ptr || !partition_bonds) return PNE_EINVAL;
    const Geometry &g = w->geo->full;
    const int NB = g.n_bonds;
    if (NB > kDtMaxBonds) {
        set_error(ctx, PNE_EINVAL, "too many bonds for the dense contraction");
        return PNE_EINVAL;
    }
    RankTerms t;
    pne_status st = rank_terms(ctx, g, rank, form, n_partitions, partition_ptr, partition_bonds, t);
    if (st) return st;
    const int n_terms = (int)t.order.size();
    std::vector<DtStep> steps;
    int64_t max_front = 1;
    st = dense_plan(ctx, g, steps, max_front);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t items = (int64_t)n_terms * w->n_sets;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(items, 2 * (int64_t)ctx->n_sm));
    DevBuf dsteps, dkind, dscr, dval;
    if ((st = dev_alloc(ctx, dsteps, steps.size() * sizeof(DtStep), s)) || (st = dev_alloc(ctx, dkind, t.kind.size(), s)) ||
        (st = dev_alloc(ctx, dscr, (size_t)grid * 2 * kDtMaxFront * 8, s)) ||
        (st = dev_alloc(ctx, dval, (size_t)items * 8, s)) ||
        (st = upload(ctx, dsteps.ptr, steps.data(), steps.size() * sizeof(DtStep), s)) ||
        (st = upload(ctx, dkind.ptr, t.kind.data(), t.kind.size(), s))) {
        dev_free(ctx, dsteps, s); dev_free(ctx, dkind, s); dev_free(ctx, dscr, s); dev_free(ctx, dval, s);
        return st;
    }
    DtParams p;
    p.steps = (const DtStep *)dsteps.ptr; p.n_steps = (int)steps.size(); p.n_bonds = NB; p.n_terms = n_terms;
    p.n_sets = w->n_sets; p.kind = (const int8_t *)dkind.ptr; p.bond_dim = g.d_bond_dim; p.rank = rank;
    p.T = (const double *)w->T.ptr; p.tens_off = g.d_tens_off; p.set_stride = g.tens_off[g.n_sites];
    p.scratch = (double *)dscr.ptr; p.value = (double *)dval.ptr;
    {
        ProfScope ps(ctx, s, "dense_terms");
        dense_term_kernel<<<grid, kDtThreads, 0, s>>>(p);
    }
    if (cudaGetLastError() != cudaSuccess) {
        dev_free(ctx, dsteps, s); dev_free(ctx, dkind, s); dev_free(ctx, dscr, s); dev_free(ctx, dval, s);
        set_error(ctx, PNE_ECUDA, "dense_term_kernel launch failed");
        return PNE_ECUDA;
    }
    std::vector<double> vals((size_t)items);
    PNE_CUDA_TRY(ctx, cudaMemcpyAsync(vals.data(), dval.ptr, vals.size() * 8, cudaMemcpyDeviceToHost, s));
    dev_free(ctx, dsteps, s); dev_free(ctx, dkind, s); dev_free(ctx, dscr, s); dev_free(ctx, dval, s);
    PNE_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const_cast<pne_weights *>(w)->last_stream = s;
    const int nops = 2 * g.n_sites + (int)std::ceil(std::log2((double)std::max<int64_t>(max_front, 2))) + t.M + 2;
    rank_results(w, form, t, vals, {}, nops, out);
    return PNE_OK;
}

pne_status pne_rank_r_expand_grid(pne_ctx *ctx, const pne_weights *w, int32_t rank, int32_t form,
                                  int32_t n_partitions, const int32_t *partition_ptr, const int32_t *partition_bonds,
                                  int32_t lx, int32_t ly, pne_dtype dtype, void *stream, pne_result *out)
{
    HostScope hs__(ctx, "rank_r_expand_grid");
    if (!ctx || !w || !out || !partition_ptr || !partition_bonds) return PNE_EINVAL;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    const Geometry &g = w->geo->full;
    if (dtype == PNE_F32) return bad("rank_r_expand_grid takes PNE_F64, PNE_TF32 or PNE_BF16");
    if (lx < 1 || ly < 1 || (int64_t)lx * ly != g.n_sites) return bad("n_sites must be lx * ly");
    RankTerms t;
    pne_status st = rank_terms(ctx, g, rank, form, n_partitions, partition_ptr, partition_bonds, t);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> vals, babs;
    if ((st = grid_term_values(ctx, w, t.kind, (int)t.order.size(), rank, lx, ly, dtype, s, vals, babs))) return st;
    const_cast<pne_weights *>(w)->last_stream = s;
    const int nops = 2 * g.n_sites + 4 * std::max(lx, ly) + t.M + 2;
    rank_results(w, form, t, vals, babs, nops, out);
    return PNE_OK;
}

pne_status pne_recursive_expand_grid(pne_ctx *ctx, const pne_weights *w, int32_t rank, int32_t n_partitions,
                                     const int32_t *partition_ptr, const int32_t *partition_bonds,
                                     int32_t n_sub_partitions, const int32_t *sub_ptr, const int32_t *sub_bonds,
                                     int32_t max_side, int32_t lx, int32_t ly, pne_dtype dtype, void *stream,
                                     pne_result *out, uint64_t *n_contractions)
{
    HostScope hs__(ctx, "recursive_expand_grid");
    if (!ctx || !w || !out || !partition_ptr || !partition_bonds || (n_sub_partitions > 0 && (!sub_ptr || !sub_bonds)))
        return PNE_EINVAL;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    const Geometry &g = w->geo->full;
    const int NB = g.n_bonds, N = g.n_sites;
    if (dtype == PNE_F32) return bad("recursive_expand_grid takes PNE_F64, PNE_TF32 or PNE_BF16");
    if (lx < 1 || ly < 1 || (int64_t)lx * ly != N) return bad("n_sites must be lx * ly");
    if (max_side < 1) return bad("max_side must be positive");
    if (n_partitions > 16) return bad("at most 16 first-level partitions");
    if (n_sub_partitions < 0 || n_sub_partitions > 64) return bad("0..64 second-level partitions");
    RankTerms t1;
    pne_status st = rank_terms(ctx, g, rank, 1, n_partitions, partition_ptr, partition_bonds, t1);
    if (st) return st;
    std::vector<std::vector<int>> sub((size_t)n_sub_partitions);
    for (int p = 0; p < n_sub_partitions; ++p) {
        if (sub_ptr[p + 1] <= sub_ptr[p] || (p == 0 && sub_ptr[0] != 0)) return bad("malformed second-level partitions");
        for (int i = sub_ptr[p]; i < sub_ptr[p + 1]; ++i) {
            const int b = sub_bonds[i];
            if (b < 0 || b >= NB) return bad("second-level partition bond out of range");
            if (rank >= g.bond_dim[b]) return bad("rank must be below every partitioned bond's dimension");
            sub[(size_t)p].push_back(b);
        }
    }
    // every first-level subset x: the cut bonds, the components left, and
    // either the sub-network itself or its expansion over the second-level
    // partitions that fit inside its too-large components
    const int n1 = (int)t1.order.size();
    std::vector<int8_t> kind;            // every network to contract
    std::vector<int> owner, sign2;       // its first-level term and second-level sign
    std::vector<int> parent((size_t)N);
    auto find = [&](int a) {
        while (parent[(size_t)a] != a) a = parent[(size_t)a] = parent[(size_t)parent[(size_t)a]];
        return a;
    };
    for (int q = 0; q < n1; ++q) {
        const int8_t *row = t1.kind.data() + (size_t)q * NB;
        for (int v = 0; v < N; ++v) parent[(size_t)v] = v;
        for (int b = 0; b < NB; ++b) {
            if (row[b] == 1) continue;
            const int ra = find(g.bond_site[2 * b]), rb = find(g.bond_site[2 * b + 1]);
            if (ra != rb) parent[(size_t)std::max(ra, rb)] = std::min(ra, rb);
        }
        // a component is too costly when both sides of its bounding box exceed max_side
        std::vector<int> x0((size_t)N, INT32_MAX), x1((size_t)N, -1), y0((size_t)N, INT32_MAX), y1((size_t)N, -1);
        for (int v = 0; v < N; ++v) {
            const size_t r = (size_t)find(v);
            x0[r] = std::min(x0[r], v % lx); x1[r] = std::max(x1[r], v % lx);
            y0[r] = std::min(y0[r], v / lx); y1[r] = std::max(y1[r], v / lx);
        }
        auto big = [&](int v) {
            const size_t r = (size_t)find(v);
            return std::min(x1[r] - x0[r] + 1, y1[r] - y0[r] + 1) > max_side;
        };
        std::vector<int> fit;
        for (int p = 0; p < n_sub_partitions; ++p) {
            bool ok = true;
            for (int b : sub[(size_t)p]) {
                const int s0 = g.bond_site[2 * b], s1 = g.bond_site[2 * b + 1];
                if (row[b] == 1 || !big(s0) || find(s0) != find(s1)) { ok = false; break; }
            }
            if (ok) fit.push_back(p);
        }
        if (fit.size() > 16) return bad("more than 16 second-level partitions fit one sub-network");
        if (fit.empty()) {
            kind.insert(kind.end(), row, row + NB);
            owner.push_back(q);
            sign2.push_back(1);
            continue;
        }
        for (uint32_t y = 1; y < (1u << fit.size()); ++y) {
            std::vector<int8_t> r2(row, row + NB);
            int k = 0;
            for (size_t i = 0; i < fit.size(); ++i)
                if (y >> i & 1) { ++k; for (int b : sub[(size_t)fit[i]]) r2[(size_t)b] = 1; }
            kind.insert(kind.end(), r2.begin(), r2.end());
            owner.push_back(q);
            sign2.push_back(k % 2 == 1 ? 1 : -1);
        }
    }
    const int nt = (int)owner.size();
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<double> vals, babs;
    if ((st = grid_term_values(ctx, w, kind, nt, rank, lx, ly, dtype, s, vals, babs))) return st;
    const_cast<pne_weights *>(w)->last_stream = s;
    // first-level values: the second-level sums (Neumaier, in network order)
    const int ns = w->n_sets;
    std::vector<double> v1((size_t)ns * n1, 0.0), b1((size_t)ns * n1, 0.0), c1((size_t)ns * n1, 0.0);
    for (int set = 0; set < ns; ++set)
        for (int i = 0; i < nt; ++i) {
            const size_t a = (size_t)set * n1 + owner[(size_t)i];
            const double x = sign2[(size_t)i] * vals[(size_t)set * nt + i], tt = v1[a] + x;
            c1[a] += (std::fabs(v1[a]) >= std::fabs(x)) ? (v1[a] - tt) + x : (x - tt) + v1[a];
            v1[a] = tt;
            b1[a] += babs[(size_t)set * nt + i];
        }
    for (size_t a = 0; a < v1.size(); ++a) v1[a] += c1[a];
    const int nops = 2 * N + 4 * std::max(lx, ly) + t1.M + 2 + 20;
    rank_results(w, 1, t1, v1, b1, nops, out);
    for (int set = 0; set < ns; ++set) out[set].n_terms = (uint64_t)nt;
    if (n_contractions) *n_contractions = (uint64_t)nt;
    return PNE_OK;
}

}  // extern "C"
