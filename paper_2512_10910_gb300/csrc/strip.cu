// Infinite-lattice strip expansion (Sec. IV.C).
//
// One uniform tensor A[l, u, r, d] on the infinite square lattice.  The BP
// fixed point of the lattice gives four messages (mR flowing +x into an l leg,
// mL flowing -x into an r leg, mD flowing +y into a u leg, mU flowing -y into
// a d leg).  A vertical strip k sites wide has the row transfer matrix
//     T_k[d_1..d_k, u_1..u_k] = sum_h mR[h_0] A[h_0,u_1,h_1,d_1] ... A[h_{k-1},u_k,h_k,d_k] mL[h_k],
// whose leading eigenvalue is lambda_k; horizontal strips are the vertical
// strips of the lattice reflected across its diagonal (A[u,l,d,r], messages
// mD, mU, mR, mL) and give gamma_k; a capped w x h patch is
// <mU^{(x)w}| T_w^h |mD^{(x)w}>.  The expansion sums the 2^(2L) - 1 subsets of
// one cell's strip partitions with signs (-1)^{|x|+1}.
//
// GPU layout.  T_k is never formed: a vector over [u_1..u_k] is pushed through
// the row one site at a time.  After j sites the running tensor is
// [d_1..d_j][h][u_{j+1}][u_{j+2}..u_k]: site j+1 maps the adjacent pair
// (h, u_{j+1}) to (d_{j+1}, h') in place, a chi^2 x chi^2 matrix applied to the
// middle axis of [P][chi^2][S] -- the same kernel for every site, with the
// capped first site (chi -> chi^2), last site (chi^2 -> chi) and one-site
// strip (chi -> chi) as its other shapes.  One thread per (p, s) keeps the
// chi^2 inputs of its fibre in registers and the matrix in shared memory (a
// broadcast read); consecutive threads take consecutive s, so the fibre's
// loads coalesce whenever S >= 32.  Every multiply-add is FP64.
//
// The power iteration keeps the vector unnormalised with a per-tensor scale;
// the reduction of each iteration forms |w|^2, <v, w> (the Rayleigh quotient
// with the unit vector v) and <mU^{(x)k}, w> (the patch of the current height)
// in one pass, per block, summed in a fixed order by the finishing kernel:
// results do not depend on the launch shape's timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pne_internal.h"

namespace pne {
namespace {

constexpr int kMaxL = PNE_STRIP_MAX_L;
constexpr int kMaxChi = PNE_STRIP_MAX_CHI;
constexpr int kThreads = 256;
constexpr int kRedBlocks = 512;                 // reduction blocks per tensor
constexpr int64_t kMaxState = (int64_t)1 << 28; // chi^(L+1) limit (2 GiB of doubles)
constexpr double kGroupBytes = 24e9;            // working set of one group of tensors

// per-tensor scalars of the running power iteration
struct IterState {
    double scale;      // v_true = scale * v_stored
    double logacc;     // ln of the norms taken out so far (patch values)
    double prev;       // ln lambda of the last iteration
    double prev_lam;   // lambda of the last iteration
    double change;     // |lambda / prev_lam - 1| of the last iteration
    int32_t iter;      // iterations done
    int32_t calm;      // successive iterations with change < tol
    int32_t done;
    int32_t status;    // 0 ok, 1 not converged, 2 degenerate
};

// per (tensor, orientation, k) record, read back at the end
struct KRecord {
    double log_lam;
    double change;
    double log_z[kMaxL + 1];
    int32_t sign_z[kMaxL + 1];
    int32_t iters;
    int32_t status;
};

// ---------------------------------------------------------------- uniform BP
// One block per tensor.  msg[n][4][chi]: mR, mL, mD, mU.
__global__ void __launch_bounds__(128) strip_bp_kernel(const double *__restrict__ A, int chi, int n, double tol,
                                                      int max_iter, double *msg, double *lz, int32_t *sweeps,
                                                      int32_t *status)
{
    const int b = blockIdx.x;
    if (b >= n) return;
    const int c4 = chi * chi * chi * chi;
    __shared__ double sA[kMaxChi * kMaxChi * kMaxChi * kMaxChi];
    __shared__ double m[4][kMaxChi], mn[4][kMaxChi];
    __shared__ double diff[4];
    __shared__ int stop;
    const double *Ab = A + (int64_t)b * c4;
    for (int i = threadIdx.x; i < c4; i += blockDim.x) sA[i] = Ab[i];
    if (threadIdx.x < 4 * chi) m[threadIdx.x / chi][threadIdx.x % chi] = rsqrt((double)chi);
    if (threadIdx.x == 0) stop = 0;
    __syncthreads();
    auto at = [&](int l, int u, int r, int d) { return sA[((l * chi + u) * chi + r) * chi + d]; };
    int it = 0;
    for (it = 1; it <= max_iter; ++it) {
        if (threadIdx.x < 4 * chi) {
            const int which = threadIdx.x / chi, i = threadIdx.x % chi;
            double acc = 0.0;
            for (int x = 0; x < chi; ++x)
                for (int y = 0; y < chi; ++y)
                    for (int z = 0; z < chi; ++z) {
                        // the three incoming messages on the legs other than the outgoing one
                        if (which == 0) acc += at(x, y, i, z) * m[0][x] * m[2][y] * m[3][z];       // mR' on r
                        else if (which == 1) acc += at(i, y, x, z) * m[1][x] * m[2][y] * m[3][z];  // mL' on l
                        else if (which == 2) acc += at(x, y, z, i) * m[0][x] * m[1][z] * m[2][y];  // mD' on d
                        else acc += at(x, i, z, y) * m[0][x] * m[1][z] * m[3][y];                  // mU' on u
                    }
            mn[which][i] = acc;
        }
        __syncthreads();
        if (threadIdx.x < 4) {
            const int w = threadIdx.x;
            double nrm = 0.0;
            int arg = 0;
            for (int i = 0; i < chi; ++i) {
                nrm += mn[w][i] * mn[w][i];
                if (fabs(mn[w][i]) > fabs(mn[w][arg])) arg = i;
            }
            const double sc = (nrm > 0.0 ? rsqrt(nrm) : 0.0) * (mn[w][arg] < 0.0 ? -1.0 : 1.0);
            double d = 0.0;
            for (int i = 0; i < chi; ++i) {
                const double x = mn[w][i] * sc;
                d = fmax(d, fabs(x - m[w][i]));
                m[w][i] = x;
            }
            diff[w] = nrm > 0.0 ? d : -1.0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const double d = fmax(fmax(diff[0], diff[1]), fmax(diff[2], diff[3]));
            stop = (diff[0] < 0 || diff[1] < 0 || diff[2] < 0 || diff[3] < 0) ? 2 : (d < tol ? 1 : 0);
        }
        __syncthreads();
        if (stop) break;
    }
    if (threadIdx.x == 0) {
        int st = stop == 2 ? 2 : (stop == 1 ? 0 : 1);
        double sh = 0.0, sv = 0.0;
        for (int i = 0; i < chi; ++i) {
            sh += m[0][i] * m[1][i];
            sv += m[2][i] * m[3][i];
        }
        if (!(fabs(sh) > 1e-300) || !(fabs(sv) > 1e-300)) st = 2;
        const double ah = st == 2 ? 1.0 : rsqrt(fabs(sh)), av = st == 2 ? 1.0 : rsqrt(fabs(sv));
        for (int i = 0; i < chi; ++i) {
            m[0][i] *= ah;
            m[1][i] *= ah * (sh < 0 ? -1.0 : 1.0);
            m[2][i] *= av;
            m[3][i] *= av * (sv < 0 ? -1.0 : 1.0);
        }
        double z = 0.0;
        for (int l = 0; l < chi; ++l)
            for (int u = 0; u < chi; ++u)
                for (int r = 0; r < chi; ++r)
                    for (int d = 0; d < chi; ++d) z += at(l, u, r, d) * m[0][l] * m[2][u] * m[1][r] * m[3][d];
        if (!(z > 0.0)) st = 2;
        lz[b] = z > 0.0 ? log(z) : 0.0;
        sweeps[b] = min(it, max_iter);
        status[b] = st;
        for (int w = 0; w < 4; ++w)
            for (int i = 0; i < chi; ++i) msg[((int64_t)b * 4 + w) * chi + i] = m[w][i];
    }
}

// ---------------------------------------------------------------- row operators
// Per (tensor, orientation): M [chi^2 x chi^2], F [chi^2 x chi], G [chi x chi^2],
// T1 [chi x chi], capTop [chi], capBot [chi].
struct OpsLayout {
    int chi;
    int64_t M, F, G, T1, top, bot, size;
    __host__ __device__ explicit OpsLayout(int c) : chi(c)
    {
        const int64_t c2 = (int64_t)c * c;
        M = 0;
        F = M + c2 * c2;
        G = F + c2 * c;
        T1 = G + c2 * c;
        top = T1 + c2;
        bot = top + c;
        size = bot + c;
    }
};

__global__ void strip_ops_kernel(const double *__restrict__ A, const double *__restrict__ msg, int chi, int n,
                                 double *ops)
{
    const int b = blockIdx.x, o = blockIdx.y;
    if (b >= n) return;
    const OpsLayout lay(chi);
    const int64_t c4 = (int64_t)chi * chi * chi * chi;
    const double *Ab = A + b * c4;
    const double *mR = msg + ((int64_t)b * 4 + 0) * chi, *mL = msg + ((int64_t)b * 4 + 1) * chi;
    const double *mD = msg + ((int64_t)b * 4 + 2) * chi, *mU = msg + ((int64_t)b * 4 + 3) * chi;
    // orientation 1: the lattice reflected across its diagonal, A'[l,u,r,d] = A[u,l,d,r]
    const double *capL = o == 0 ? mR : mD, *capR = o == 0 ? mL : mU;
    const double *capT = o == 0 ? mD : mR, *capB = o == 0 ? mU : mL;
    double *out = ops + ((int64_t)b * 2 + o) * lay.size;
    auto Ao = [&](int l, int u, int r, int d) {
        return o == 0 ? Ab[((l * chi + u) * chi + r) * chi + d] : Ab[((u * chi + l) * chi + d) * chi + r];
    };
    const int c2 = chi * chi;
    for (int i = threadIdx.x; i < c2 * c2; i += blockDim.x) {
        const int row = i / c2, col = i % c2;          // row (d, h'), col (h, u)
        out[lay.M + i] = Ao(col / chi, col % chi, row % chi, row / chi);
    }
    for (int i = threadIdx.x; i < c2 * chi; i += blockDim.x) {
        const int row = i / chi, u = i % chi;          // F: row (d, h'), col u
        double acc = 0.0;
        for (int h = 0; h < chi; ++h) acc += capL[h] * Ao(h, u, row % chi, row / chi);
        out[lay.F + i] = acc;
        const int d = i / c2, col = i % c2;            // G: row d, col (h, u)
        double g = 0.0;
        for (int hp = 0; hp < chi; ++hp) g += Ao(col / chi, col % chi, hp, d) * capR[hp];
        out[lay.G + i] = g;
    }
    for (int i = threadIdx.x; i < c2; i += blockDim.x) {
        const int d = i / chi, u = i % chi;
        double acc = 0.0;
        for (int h = 0; h < chi; ++h)
            for (int hp = 0; hp < chi; ++hp) acc += capL[h] * Ao(h, u, hp, d) * capR[hp];
        out[lay.T1 + i] = acc;
    }
    for (int i = threadIdx.x; i < chi; i += blockDim.x) {
        out[lay.top + i] = capT[i];
        out[lay.bot + i] = capB[i];
    }
}

// ---------------------------------------------------------------- power iteration
struct ApplyParams {
    const double *in;
    double *out;
    int64_t in_stride, out_stride;   // elements between tensors in the two buffers
    const double *ops;       // [n][2][size]
    int64_t ops_stride;      // elements between tensors in ops (2 * size)
    int64_t mat_off;         // orientation * size + matrix offset
    int use_scale;           // multiply the input by the tensor's iteration scale
    const IterState *st;
    int64_t P, S;
};

// out[p][o][s] = sum_i mat[o][i] * in[p][i][s] (* scale): one site of the row.
// IN / OUT formats: 0 FP64, 1 float-float pair (hi, lo) in the same 8 bytes.
// With FF the multiply-adds run on the FP32 pipes as compensated dot products
// (each product split exactly by one FMA, the running sum by Knuth's two-sum,
// the error terms and the low-part cross products gathered in one FP32
// compensation): about 2^-48 relative to sum |a x| per output, where the FP64
// pipe of this part retires 1/60 of the FP32 rate.
struct ffp { float h, l; };

__device__ __forceinline__ ffp split_double(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}

template <int NIN, int NOUT, int IN_FF, int OUT_FF>
__global__ void __launch_bounds__(kThreads) strip_apply_kernel(ApplyParams p)
{
    const int b = blockIdx.y;
    if (p.st[b].done) return;
    constexpr bool FF = IN_FF || OUT_FF;
    __shared__ double M[FF ? 1 : NOUT * NIN];
    __shared__ float Mh[FF ? NOUT * NIN : 1], Ml[FF ? NOUT * NIN : 1];
    const double *mat = p.ops + b * p.ops_stride + p.mat_off;
    for (int i = threadIdx.x; i < NOUT * NIN; i += blockDim.x) {
        if (FF) {
            const ffp a = split_double(mat[i]);
            Mh[i] = a.h;
            Ml[i] = a.l;
        } else {
            M[i] = mat[i];
        }
    }
    __syncthreads();
    const double sc = p.use_scale ? p.st[b].scale : 1.0;
    const int64_t units = p.P * p.S;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < units; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pp = q / p.S, s = q - pp * p.S;
        const int64_t src0 = (pp * NIN) * p.S + s, dst0 = (pp * NOUT) * p.S + s;
        if (!FF) {
            const double *in = p.in + b * p.in_stride + src0;
            double *out = p.out + b * p.out_stride + dst0;
            double x[NIN];
#pragma unroll
            for (int i = 0; i < NIN; ++i) x[i] = __ldg(in + i * p.S) * sc;
#pragma unroll 4
            for (int o = 0; o < NOUT; ++o) {
                double acc = 0.0;
#pragma unroll
                for (int i = 0; i < NIN; ++i) acc = fma(M[o * NIN + i], x[i], acc);
                out[o * p.S] = acc;
            }
        } else {
            float xh[NIN], xl[NIN];
            if (IN_FF) {
                const float2 *in = reinterpret_cast<const float2 *>(p.in + b * p.in_stride) + src0;
#pragma unroll
                for (int i = 0; i < NIN; ++i) {
                    const float2 v = __ldg(in + i * p.S);
                    xh[i] = v.x;
                    xl[i] = v.y;
                }
            } else {
                const double *in = p.in + b * p.in_stride + src0;
#pragma unroll
                for (int i = 0; i < NIN; ++i) {
                    const ffp v = split_double(__ldg(in + i * p.S) * sc);
                    xh[i] = v.h;
                    xl[i] = v.l;
                }
            }
#pragma unroll 2
            for (int o = 0; o < NOUT; ++o) {
                float sh = 0.f, c = 0.f;
#pragma unroll
                for (int i = 0; i < NIN; ++i) {
                    const float ah = Mh[o * NIN + i], al = Ml[o * NIN + i];
                    const float pr = __fmul_rn(ah, xh[i]);
                    const float e = __fmaf_rn(ah, xh[i], -pr);
                    const float t = __fadd_rn(sh, pr);
                    const float bb = __fsub_rn(t, sh);
                    const float q2 = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(pr, bb));
                    sh = t;
                    c = __fadd_rn(c, __fadd_rn(q2, e));
                    c = __fmaf_rn(ah, xl[i], c);
                    c = __fmaf_rn(al, xh[i], c);
                }
                const float hi = __fadd_rn(sh, c);
                const float lo = __fsub_rn(c, __fsub_rn(hi, sh));
                if (OUT_FF) {
                    float2 *out = reinterpret_cast<float2 *>(p.out + b * p.out_stride) + dst0;
                    out[o * p.S] = make_float2(hi, lo);
                } else {
                    double *out = p.out + b * p.out_stride + dst0;
                    out[o * p.S] = (double)hi + (double)lo;
                }
            }
        }
    }
}

// v = capTop^{(x)k}; scalars reset
__global__ void strip_init_kernel(double *V, int64_t stride, const double *ops, int64_t ops_stride, int64_t top_off,
                                  int chi, int k, int64_t N, IterState *st, int n)
{
    const int b = blockIdx.y;
    if (b >= n) return;
    const double *top = ops + b * ops_stride + top_off;
    double *v = V + b * stride;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        int64_t r = q;
        double x = 1.0;
        for (int i = 0; i < k; ++i) {
            x *= top[r % chi];
            r /= chi;
        }
        v[q] = x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double nt = 0.0;
        for (int i = 0; i < chi; ++i) nt += top[i] * top[i];
        nt = sqrt(nt);
        IterState s;
        s.scale = pow(nt, -(double)k);
        s.logacc = k * log(nt);
        s.prev = 0.0;
        s.prev_lam = 0.0;
        s.change = INFINITY;
        s.iter = 0;
        s.calm = 0;
        s.done = 0;
        s.status = 0;
        st[b] = s;
    }
}

__device__ __forceinline__ void block_sum3(double &a, double &b, double &c, double *sh)
{
    for (int off = 16; off > 0; off >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, off);
        b += __shfl_xor_sync(0xffffffffu, b, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (lane == 0) {
        sh[3 * w] = a;
        sh[3 * w + 1] = b;
        sh[3 * w + 2] = c;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < nw; ++i) {
            a += sh[3 * i];
            b += sh[3 * i + 1];
            c += sh[3 * i + 2];
        }
    }
}

// per block: sum w^2, sum v w, sum w * capBot^{(x)k}.  The cap product of an
// index is looked up per group of g base-chi digits (chi^g <= 256 entries, a
// shorter table for the last r = k mod g digits): a few FP64 multiplies per
// entry instead of k.
__global__ void __launch_bounds__(kThreads) strip_reduce_kernel(const double *V, const double *W, int64_t stride,
                                                                const double *ops, int64_t ops_stride,
                                                                int64_t bot_off, int chi, int k, int64_t N,
                                                                const IterState *st, double *part)
{
    const int b = blockIdx.y;
    if (st[b].done) return;
    __shared__ double sh[3 * (kThreads / 32)];
    __shared__ double bot[kMaxChi];
    __shared__ double tabF[256], tabP[256];
    int g = 1, cg = chi;
    while (cg * chi <= 256) {
        cg *= chi;
        ++g;
    }
    const int ng = k / g, r = k - ng * g;
    int cr = 1;
    for (int i = 0; i < r; ++i) cr *= chi;
    if (threadIdx.x < chi) bot[threadIdx.x] = ops[b * ops_stride + bot_off + threadIdx.x];
    __syncthreads();
    for (int j = threadIdx.x; j < cg; j += blockDim.x) {
        double x = 1.0;
        int t = j;
        for (int i = 0; i < g; ++i) {
            x *= bot[t % chi];
            t /= chi;
        }
        tabF[j] = x;
        if (j < cr) {
            double y = 1.0;
            t = j;
            for (int i = 0; i < r; ++i) {
                y *= bot[t % chi];
                t /= chi;
            }
            tabP[j] = y;
        }
    }
    __syncthreads();
    const double *v = V + b * stride, *w = W + b * stride;
    double ww = 0.0, vw = 0.0, wc = 0.0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (int64_t)gridDim.x * blockDim.x) {
        const double x = w[q];
        ww = fma(x, x, ww);
        vw = fma(v[q], x, vw);
        int64_t t = q;
        double c = r ? tabP[t % cr] : 1.0;
        if (r) t /= cr;
        for (int i = 0; i < ng; ++i) {
            c *= tabF[t % cg];
            t /= cg;
        }
        wc = fma(x, c, wc);
    }
    block_sum3(ww, vw, wc, sh);
    if (threadIdx.x == 0) {
        double *o = part + ((int64_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = ww;
        o[1] = vw;
        o[2] = wc;
    }
}

__global__ void strip_finish_kernel(const double *part, int nblk, IterState *st, KRecord *rec, int64_t rec_stride,
                                    int L, double tol, int max_iter, int n)
{
    const int b = blockIdx.x;
    if (b >= n || st[b].done) return;
    __shared__ double sh[3 * (kThreads / 32)];
    double ww = 0.0, vw = 0.0, wc = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        const double *o = part + ((int64_t)b * nblk + i) * 3;
        ww += o[0];
        vw += o[1];
        wc += o[2];
    }
    block_sum3(ww, vw, wc, sh);
    if (threadIdx.x != 0) return;
    IterState s = st[b];
    KRecord &r = rec[b * rec_stride];
    const int h = s.iter + 1;
    if (h <= L) {
        r.log_z[h] = s.logacc + log(fabs(wc));
        r.sign_z[h] = wc > 0.0 ? 1 : (wc < 0.0 ? -1 : 0);
    }
    const double lam = s.scale * vw;
    const double nw = sqrt(ww);
    s.logacc += log(nw);
    s.scale = 1.0 / nw;
    s.iter = h;
    if (!(lam > 0.0) || !(nw > 0.0) || !isfinite(lam)) {
        s.status = 2;
        s.done = 1;
    } else {
        // relative change of lambda itself (ln lambda ~ k ln z would quantise
        // the difference to its own ulp)
        s.change = h > 1 ? fabs(lam / s.prev_lam - 1.0) : INFINITY;
        s.prev_lam = lam;
        s.prev = log(lam);
        s.calm = s.change < tol ? s.calm + 1 : 0;
        if (h >= L && s.calm >= 3) s.done = 1;
        else if (h >= max_iter) {
            s.done = 1;
            s.status = 1;
        }
    }
    r.log_lam = s.prev;
    r.change = s.change;
    r.iters = s.iter;
    r.status = s.status;
    st[b] = s;
}

// ---------------------------------------------------------------- the subset sum
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

struct DD {
    double hi = 0.0, lo = 0.0;
    __device__ __forceinline__ void add(double x)
    {
        double s, e;
        two_sum(hi, x, s, e);
        e += lo;
        hi = s + e;
        lo = e - (hi - s);
    }
    __device__ __forceinline__ void add(DD y)
    {
        double s, e;
        two_sum(hi, y.hi, s, e);
        e += lo + y.lo;
        hi = s + e;
        lo = e - (hi - s);
    }
};

// the gaps between the set bits of a cyclic L-bit mask (at most L of them)
__device__ __forceinline__ int mask_gaps(uint32_t m, int L, int *g)
{
    const int first = __ffs(m) - 1;
    int prev = first, n = 0;
    uint32_t rest = m & (m - 1);
    while (rest) {
        const int o = __ffs(rest) - 1;
        g[n++] = o - prev;
        prev = o;
        rest &= rest - 1;
    }
    g[n++] = L - prev + first;
    return n;
}

struct SumParams {
    const KRecord *rec;      // [n][2][kMaxL + 1]
    const double *lz_bp;     // [n]
    int L, two_d, n;
    double *part;            // [n][nblk][3]: hi, lo, signed count
};

// 2D: block per vertical mask V, threads over horizontal masks H.
// 1D: thread per vertical mask.
__global__ void __launch_bounds__(kThreads) strip_sum_kernel(SumParams p)
{
    const int b = blockIdx.y;
    const int L = p.L;
    const uint32_t full = 1u << L;
    const KRecord *rv = p.rec + ((int64_t)b * 2 + 0) * (kMaxL + 1);
    const KRecord *rh = p.rec + ((int64_t)b * 2 + 1) * (kMaxL + 1);
    const double ref = (p.two_d ? (double)L * L : (double)L) * p.lz_bp[b];
    DD acc;
    double count = 0.0;
    __shared__ double cV[kMaxL + 1];
    __shared__ int sV[kMaxL + 1];
    __shared__ double lamV;
    int g[kMaxL];
    if (p.two_d) {
        const uint32_t V = blockIdx.x;
        if (threadIdx.x == 0) {
            int gv[kMaxL];
            const int nv = V ? mask_gaps(V, L, gv) : 0;
            double lv = 0.0;
            for (int i = 0; i < nv; ++i) lv += rv[gv[i]].log_lam;
            lamV = L * lv;
            for (int h = 1; h <= L; ++h) {
                double c = 0.0;
                int sg = 1;
                for (int i = 0; i < nv; ++i) {
                    c += rv[gv[i]].log_z[h];
                    sg *= rv[gv[i]].sign_z[h];
                }
                cV[h] = c;
                sV[h] = sg;
            }
        }
        __syncthreads();
        for (uint32_t H = threadIdx.x; H < full; H += blockDim.x) {
            if (V == 0 && H == 0) continue;
            double t;
            int sg = 1;
            if (H == 0) {
                t = lamV;
            } else {
                const int nh = mask_gaps(H, L, g);
                t = 0.0;
                if (V == 0) {
                    for (int i = 0; i < nh; ++i) t += rh[g[i]].log_lam;
                    t *= L;
                } else {
                    for (int i = 0; i < nh; ++i) {
                        t += cV[g[i]];
                        sg *= sV[g[i]];
                    }
                }
            }
            const int s = ((__popc(V) + __popc(H)) & 1) ? sg : -sg;
            if (s == 0) continue;
            acc.add(s * expm1(t - ref));
            count += s;
        }
    } else {
        const uint32_t V = blockIdx.x * blockDim.x + threadIdx.x;
        if (V >= 1 && V < full) {
            const int nv = mask_gaps(V, L, g);
            double t = 0.0;
            for (int i = 0; i < nv; ++i) t += rv[g[i]].log_lam;
            const int s = (__popc(V) & 1) ? 1 : -1;
            acc.add(s * expm1(t - ref));
            count += s;
        }
    }
    // block reduction in double-double, fixed order
    __shared__ double sh[3 * kThreads];
    sh[3 * threadIdx.x] = acc.hi;
    sh[3 * threadIdx.x + 1] = acc.lo;
    sh[3 * threadIdx.x + 2] = count;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            DD a;
            a.hi = sh[3 * threadIdx.x];
            a.lo = sh[3 * threadIdx.x + 1];
            DD c;
            c.hi = sh[3 * (threadIdx.x + off)];
            c.lo = sh[3 * (threadIdx.x + off) + 1];
            a.add(c);
            sh[3 * threadIdx.x] = a.hi;
            sh[3 * threadIdx.x + 1] = a.lo;
            sh[3 * threadIdx.x + 2] += sh[3 * (threadIdx.x + off) + 2];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double *o = p.part + ((int64_t)b * gridDim.x + blockIdx.x) * 3;
        o[0] = sh[0];
        o[1] = sh[1];
        o[2] = sh[2];
    }
}

// f per tensor from the block partials: f = -(ref + ln(count + sum)) / cell
__global__ void strip_sum_finish_kernel(const double *part, int nblk, const double *lz_bp, int L, int two_d, int n,
                                        double *f, int32_t *status)
{
    const int b = blockIdx.x;
    if (b >= n || threadIdx.x != 0) return;
    DD acc;
    double count = 0.0;
    for (int i = 0; i < nblk; ++i) {
        const double *o = part + ((int64_t)b * nblk + i) * 3;
        DD y;
        y.hi = o[0];
        y.lo = o[1];
        acc.add(y);
        count += o[2];
    }
    const double cell = two_d ? (double)L * L : (double)L;
    const double ref = cell * lz_bp[b];
    // ln(count + hi + lo); with count == 1 (positive pieces) through log1p
    const double rest = (count - 1.0) + acc.hi + acc.lo;
    if (!(1.0 + rest > 0.0)) {
        f[b] = NAN;
        status[b] = 2;
        return;
    }
    f[b] = -(ref + log1p(rest)) / cell;
    status[b] = 0;
}

template <int NIN, int NOUT, int IN_FF, int OUT_FF>
cudaError_t launch_apply(const ApplyParams &p, int n, cudaStream_t s)
{
    const int64_t units = p.P * p.S;
    int64_t blocks = (units + kThreads - 1) / kThreads;
    blocks = std::min<int64_t>(std::max<int64_t>(blocks, 1), 152 * 16);
    strip_apply_kernel<NIN, NOUT, IN_FF, OUT_FF><<<dim3((unsigned)blocks, (unsigned)n), kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

// shape 0 one-site strip, 1 first site, 2 middle site, 3 last site; ff: the
// running tensor between the first and the last site is float-float
template <int CHI>
cudaError_t apply_shape(int shape, int ff, const ApplyParams &p, int n, cudaStream_t s)
{
    constexpr int C2 = CHI * CHI;
    switch (shape) {
    case 0: return launch_apply<CHI, CHI, 0, 0>(p, n, s);
    case 1: return ff ? launch_apply<CHI, C2, 0, 1>(p, n, s) : launch_apply<CHI, C2, 0, 0>(p, n, s);
    case 2: return ff ? launch_apply<C2, C2, 1, 1>(p, n, s) : launch_apply<C2, C2, 0, 0>(p, n, s);
    default: return ff ? launch_apply<C2, CHI, 1, 0>(p, n, s) : launch_apply<C2, CHI, 0, 0>(p, n, s);
    }
}

cudaError_t apply_site(int chi, int shape, int ff, const ApplyParams &p, int n, cudaStream_t s)
{
    switch (chi) {
    case 2: return apply_shape<2>(shape, ff, p, n, s);
    case 3: return apply_shape<3>(shape, ff, p, n, s);
    case 4: return apply_shape<4>(shape, ff, p, n, s);
    case 5: return apply_shape<5>(shape, ff, p, n, s);
    case 6: return apply_shape<6>(shape, ff, p, n, s);
    case 7: return apply_shape<7>(shape, ff, p, n, s);
    default: return apply_shape<8>(shape, ff, p, n, s);
    }
}

}  // namespace
}  // namespace pne

using namespace pne;

extern "C" {

pne_status pne_strip_expansion(pne_ctx *ctx, int32_t chi, int32_t n_tensors, const double *A, int32_t A_on_device,
                               const pne_strip_opts *opts, void *stream, pne_strip_result *out)
{
    HostScope hs__(ctx, "strip_expansion");
    if (!ctx || !A || !opts || !out) return PNE_EINVAL;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    const int L = opts->L;
    if (chi < 2 || chi > kMaxChi) return bad("chi must be in 2 .. PNE_STRIP_MAX_CHI");
    if (n_tensors < 1 || n_tensors > 65535) return bad("n_tensors must be in 1 .. 65535");
    if (L < 1 || L > kMaxL) return bad("L must be in 1 .. PNE_STRIP_MAX_L");
    std::vector<int64_t> cpow(L + 2, 1);
    for (int i = 1; i <= L + 1; ++i) cpow[i] = cpow[i - 1] * chi;
    const int64_t state = cpow[L + 1], vec_max = cpow[L];
    if (state > kMaxState) return bad("chi^(L+1) exceeds 2^28");
    const int two_d = opts->two_d ? 1 : 0;
    const double bp_tol = opts->bp_tol > 0 ? opts->bp_tol : 1e-14;
    const double eig_tol = opts->eig_tol > 0 ? opts->eig_tol : 1e-14;
    const int bp_max = opts->bp_max_iter > 0 ? opts->bp_max_iter : 100000;
    const int eig_max = std::max(L, opts->eig_max_iter > 0 ? opts->eig_max_iter : 20000);
    if (opts->arithmetic != 0 && opts->arithmetic != 1) return bad("arithmetic must be 0 (FP64) or 1 (float-float)");
    const int ff = opts->arithmetic;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = n_tensors;
    const OpsLayout lay(chi);
    const int64_t c4 = (int64_t)chi * chi * chi * chi;
    // tensors per group: 2 chi^L + 2 chi^(L+1) doubles each
    const double per = 8.0 * (2.0 * vec_max + 2.0 * state);
    const int group = (int)std::max<double>(1.0, std::min<double>({(double)n, 4096.0, std::floor(kGroupBytes / per)}));
    const int64_t rec_per = 2 * (kMaxL + 1);     // records per tensor

    DevBuf dA, dMsg, dScal, dOps, dBuf, dSt, dRec, dPart, dF;
    auto cleanup = [&]() {
        for (DevBuf *b : {&dA, &dMsg, &dScal, &dOps, &dBuf, &dSt, &dRec, &dPart, &dF}) dev_free(ctx, *b, s);
    };
    const int64_t sum_blocks = two_d ? (int64_t)1 << L : std::max<int64_t>(1, ((1LL << L) + kThreads - 1) / kThreads);
    const size_t part_elems = std::max<size_t>((size_t)group * kRedBlocks * 3, (size_t)n * sum_blocks * 3);
    pne_status st;
    if ((st = dev_alloc(ctx, dA, (size_t)n * c4 * 8, s)) || (st = dev_alloc(ctx, dMsg, (size_t)n * 4 * chi * 8, s)) ||
        (st = dev_alloc(ctx, dScal, (size_t)n * 16, s)) || (st = dev_alloc(ctx, dOps, (size_t)n * 2 * lay.size * 8, s)) ||
        (st = dev_alloc(ctx, dBuf, (size_t)group * (2 * vec_max + 2 * state) * 8, s)) ||
        (st = dev_alloc(ctx, dSt, (size_t)group * sizeof(IterState), s)) ||
        (st = dev_alloc(ctx, dRec, (size_t)n * rec_per * sizeof(KRecord), s)) ||
        (st = dev_alloc(ctx, dPart, part_elems * 8, s)) || (st = dev_alloc(ctx, dF, (size_t)n * 16, s))) {
        cleanup();
        return st;
    }
    auto cuda_fail = [&](cudaError_t e, const char *what) {
        set_error(ctx, PNE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
        cleanup();
        return PNE_ECUDA;
    };
    cudaError_t e = cudaMemcpyAsync(dA.ptr, A, (size_t)n * c4 * 8,
                                    A_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "upload of the tensors");
    if ((e = cudaMemsetAsync(dRec.ptr, 0, (size_t)n * rec_per * sizeof(KRecord), s)) != cudaSuccess)
        return cuda_fail(e, "record clear");
    double *lz = (double *)dScal.ptr;
    int32_t *sweeps = (int32_t *)(lz + n), *bp_status = sweeps + n;
    {
        ProfScope ps(ctx, s, "strip_bp");
        strip_bp_kernel<<<n, 128, 0, s>>>((const double *)dA.ptr, chi, n, bp_tol, bp_max, (double *)dMsg.ptr, lz,
                                          sweeps, bp_status);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_bp_kernel");
    {
        ProfScope ps(ctx, s, "strip_ops");
        strip_ops_kernel<<<dim3(n, 2), 128, 0, s>>>((const double *)dA.ptr, (const double *)dMsg.ptr, chi, n,
                                                    (double *)dOps.ptr);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_ops_kernel");
    std::vector<char> hb((size_t)n * 16);
    if ((e = cudaMemcpyAsync(hb.data(), lz, (size_t)n * 16, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "BP record");
    const double *h_lz = (const double *)hb.data();
    const int32_t *h_sweeps = (const int32_t *)(h_lz + n), *h_bpst = h_sweeps + n;
    for (int b = 0; b < n; ++b) {
        if (h_bpst[b] == 2) {
            std::vector<double> hm((size_t)4 * chi);
            cudaMemcpy(hm.data(), (const double *)dMsg.ptr + (size_t)b * 4 * chi, hm.size() * 8, cudaMemcpyDeviceToHost);
            std::string msg = "uniform BP of tensor " + std::to_string(b) + ": a message, a message overlap or z_BP vanished"
                              " (after " + std::to_string(h_sweeps[b]) + " sweeps; messages";
            for (double x : hm) msg += " " + std::to_string(x);
            set_error(ctx, PNE_EDEGENERATE, msg + ")");
            cleanup();
            return PNE_EDEGENERATE;
        }
    }

    double *bufV = (double *)dBuf.ptr;
    double *bufW = bufV + (size_t)group * vec_max;
    double *bufX = bufW + (size_t)group * vec_max, *bufY = bufX + (size_t)group * state;
    IterState *dst = (IterState *)dSt.ptr;
    KRecord *drec = (KRecord *)dRec.ptr;
    double *part = (double *)dPart.ptr;
    std::vector<IterState> h_state(group);
    const int64_t ops_stride = 2 * lay.size;

    for (int g0 = 0; g0 < n; g0 += group) {
        const int gn = std::min(group, n - g0);
        const double *ops_g = (const double *)dOps.ptr + (size_t)g0 * ops_stride;
        for (int o = 0; o < 1 + two_d; ++o) {
            const int64_t orient = (int64_t)o * lay.size;
            for (int k = 1; k <= L; ++k) {
                const int64_t N = cpow[k];
                double *V = bufV, *W = bufW;
                {
                    const int64_t blocks = std::min<int64_t>((N + kThreads - 1) / kThreads, 152 * 8);
                    ProfScope ps(ctx, s, "strip_init");
                    strip_init_kernel<<<dim3((unsigned)blocks, gn), kThreads, 0, s>>>(
                        V, vec_max, ops_g, ops_stride, orient + lay.top, chi, k, N, dst, gn);
                }
                if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_init_kernel");
                KRecord *rec_k = drec + (size_t)g0 * rec_per + o * (kMaxL + 1) + k;
                const int check_every = N >= (1 << 16) ? 1 : (N >= (1 << 10) ? 4 : 16);
                const int64_t rb = std::min<int64_t>(kRedBlocks, (N + kThreads - 1) / kThreads);
                for (int it = 0; it < eig_max; ++it) {
                    {
                        ProfScope ps(ctx, s, "strip_row");
                        ApplyParams ap;
                        ap.ops = ops_g;
                        ap.ops_stride = ops_stride;
                        ap.st = dst;
                        if (k == 1) {
                            ap.in = V; ap.out = W;
                            ap.in_stride = ap.out_stride = vec_max;
                            ap.mat_off = orient + lay.T1;
                            ap.use_scale = 1;
                            ap.P = 1; ap.S = 1;
                            if ((e = apply_site(chi, 0, 0, ap, gn, s)) != cudaSuccess) return cuda_fail(e, "strip_apply");
                        } else {
                            // site j maps [chi^j][pair][chi^(k-1-j)]; V -> X -> Y -> X ... -> W
                            const double *cur = V;
                            int64_t cur_stride = vec_max;
                            for (int j = 0; j < k; ++j) {
                                const bool last = j == k - 1;
                                double *nxt = last ? W : ((j & 1) ? bufY : bufX);
                                ap.in = cur;
                                ap.out = nxt;
                                ap.in_stride = cur_stride;
                                ap.out_stride = last ? vec_max : state;
                                ap.use_scale = j == 0;
                                ap.P = cpow[j];
                                ap.S = cpow[k - 1 - j];
                                const int shape = j == 0 ? 1 : (last ? 3 : 2);
                                ap.mat_off = orient + (j == 0 ? lay.F : (last ? lay.G : lay.M));
                                if ((e = apply_site(chi, shape, ff, ap, gn, s)) != cudaSuccess)
                                    return cuda_fail(e, "strip_apply");
                                cur = nxt;
                                cur_stride = ap.out_stride;
                            }
                        }
                    }
                    {
                        ProfScope ps(ctx, s, "strip_reduce");
                        strip_reduce_kernel<<<dim3((unsigned)rb, gn), kThreads, 0, s>>>(
                            V, W, vec_max, ops_g, ops_stride, orient + lay.bot, chi, k, N, dst, part);
                        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_reduce_kernel");
                        strip_finish_kernel<<<gn, kThreads, 0, s>>>(part, (int)rb, dst, rec_k, rec_per, L, eig_tol,
                                                                    eig_max, gn);
                        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_finish_kernel");
                    }
                    std::swap(V, W);
                    if ((it + 1) % check_every == 0 || it + 1 == eig_max) {
                        if ((e = cudaMemcpyAsync(h_state.data(), dst, (size_t)gn * sizeof(IterState),
                                                 cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
                            (e = cudaStreamSynchronize(s)) != cudaSuccess)
                            return cuda_fail(e, "power iteration state");
                        bool all = true;
                        for (int b = 0; b < gn; ++b) all = all && h_state[b].done;
                        if (all) break;
                    }
                }
            }
        }
    }

    // the subset sum, every tensor at once
    SumParams sp;
    sp.rec = drec;
    sp.lz_bp = lz;
    sp.L = L;
    sp.two_d = two_d;
    sp.n = n;
    sp.part = part;
    double *df = (double *)dF.ptr;
    int32_t *dfs = (int32_t *)(df + n);
    {
        ProfScope ps(ctx, s, "strip_sum");
        strip_sum_kernel<<<dim3((unsigned)sum_blocks, n), kThreads, 0, s>>>(sp);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_sum_kernel");
        strip_sum_finish_kernel<<<n, 32, 0, s>>>(part, (int)sum_blocks, lz, L, two_d, n, df, dfs);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "strip_sum_finish_kernel");
    }
    std::vector<KRecord> hrec((size_t)n * rec_per);
    std::vector<double> hmsg((size_t)n * 4 * chi);
    std::vector<char> hf((size_t)n * 16);
    if ((e = cudaMemcpyAsync(hrec.data(), drec, hrec.size() * sizeof(KRecord), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hmsg.data(), dMsg.ptr, hmsg.size() * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hf.data(), df, hf.size(), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "strip results");
    cleanup();
    const double *h_f = (const double *)hf.data();
    const int32_t *h_fs = (const int32_t *)(h_f + n);
    pne_status worst = PNE_OK;
    for (int b = 0; b < n; ++b) {
        pne_strip_result &r = out[b];
        std::memset(&r, 0, sizeof(r));
        r.f = h_f[b];
        r.f_bp = -h_lz[b];
        r.bp_sweeps = h_sweeps[b];
        pne_status sb = h_bpst[b] == 1 ? PNE_ENOCONV : PNE_OK;
        r.eig_change = 0.0;
        for (int o = 0; o < 1 + two_d; ++o)
            for (int k = 1; k <= L; ++k) {
                const KRecord &kr = hrec[(size_t)b * rec_per + o * (kMaxL + 1) + k];
                (o == 0 ? r.log_lambda : r.log_gamma)[k] = kr.log_lam;
                r.eig_change = std::max(r.eig_change, kr.change);
                r.eig_iters = std::max(r.eig_iters, kr.iters);
                r.iters[o * (kMaxL + 1) + k] = kr.iters;
                if (kr.status == 2) sb = PNE_EDEGENERATE;
                else if (kr.status == 1 && sb == PNE_OK) sb = PNE_ENOCONV;
                if (o == 0)
                    for (int h = 1; h <= L; ++h) {
                        r.log_z[k * (kMaxL + 1) + h] = kr.log_z[h];
                        r.sign_z[k * (kMaxL + 1) + h] = kr.sign_z[h];
                    }
            }
        if (h_fs[b] == 2) sb = PNE_EDEGENERATE;
        for (int i = 0; i < 4 * chi; ++i) r.messages[(i / chi) * kMaxChi + i % chi] = hmsg[(size_t)b * 4 * chi + i];
        r.status = sb;
        if (sb == PNE_EDEGENERATE || (sb == PNE_ENOCONV && worst == PNE_OK)) worst = sb;
    }
    if (worst != PNE_OK)
        set_error(ctx, worst, worst == PNE_ENOCONV ? "strip expansion: BP or a power iteration did not converge"
                                                   : "strip expansion: an eigenvalue, a patch sum or the total is not positive");
    return worst;
}

}  // extern "C"
