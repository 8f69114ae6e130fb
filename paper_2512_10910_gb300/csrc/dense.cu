// Dense contractions of blocked large-chi networks on the tensor cores
// (tcgen05), and the exact contraction of 2D grid networks built on them.
//
// The paper's own benchmarks group patches of the lattice into single tensors
// of bond dimension chi = 16 or 64 (App. A) and contract the resulting small
// networks exactly (Sec. III, IV.A).  At such bond dimensions the exact
// contraction is a chain of dense matrix products: a 2D grid contracted row
// by row keeps a running tensor over the open legs, and absorbing one site is
//     out[rest][d][h'] = sum_{u,h} in[u][rest][h] * T[h, u, h', d],
// a GEMM with M = |rest| (up to chi^(w-1) for width w), K = chi_u chi_h and
// N = chi_d chi_h' (256 each at chi = 16).  The running tensor is kept in a
// "ring" order -- the legs still to be contracted from above first, then the
// legs already produced, then the horizontal leg -- so the site's two input
// legs sit at the two ends and its two output legs are appended at the end:
// the next site finds its own legs at the ends again, across rows too.
//
// The GEMM (tc_gemm_kernel): one CTA per 128 x BN tile of the output (BN <= 256)
// and tensor set.  K is staged 128 bytes per row at a time (32 TF32 or 64 BF16
// values) in two shared-memory stages, written by all threads in the
// canonical no-swizzle K-major layout (8-row x 16-byte core matrices, the two
// core matrices of one MMA K step 128 bytes apart, 8-row groups 1024 bytes
// apart); one elected thread issues tcgen05.mma (M = 128, N = BN, FP32
// accumulation in tensor memory) and commits each stage to an mbarrier, which
// the loaders wait on (bounded) before refilling the stage.  The epilogue
// reads the accumulator with tcgen05.ld (a warp per 32 lanes = rows) and
// records the largest |entry| per set, from which the next step takes a
// power-of-two scale (kept exactly in a log-2 counter).  The FP64 form
// (f64_gemm_kernel) is a plain tiled GEMM on the CUDA cores with the same
// interface: the reference the reduced-precision forms are stated against.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "pne_internal.h"

namespace pne {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTcBM = 128;
constexpr int kChunk = 128;                   // K bytes per row per stage
constexpr int kATileBytes = kTcBM * kChunk;   // 16 KB
constexpr int kTmaChunk = 64;                 // K bytes per row per stage of the TMA-fed kernel
constexpr uint64_t kWaitNs = 2000000000ull;   // bounded mbarrier waits: 2 s

// ---------------------------------------------------------------- PTX wrappers
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading (K) and stride (M/N)
// byte offsets between core matrices, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor: FP32 accumulator, A and B of one format (2 = TF32
// for kind::tf32, 1 = BF16 for kind::f16), both K-major, M and N
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem), "r"(ncols)
                 : "memory");
}
__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_after()
{
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before()
{
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
template <int EB>
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if (EB == 4)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc)
                     : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t addr, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(addr), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// bounded wait (about two seconds of the global timer); false when it gave up
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    const uint64_t t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(addr, parity)) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t to_tf32(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// ---------------------------------------------------------------- the GEMMs
// C[b][m][n] = sum_k A[b][m][k] B[b][n][k]  (A and B K-major, C row-major)
template <typename T>
struct GemmParams {
    const T *A;
    int64_t lda, strideA;
    const T *B;
    int64_t ldb, strideB;
    T *C;
    int64_t ldc, strideC;
    int M, N, K;
    unsigned long long *maxbits;   // [batch]: largest |C| (bit pattern, atomicMax), or nullptr
    int *err;                      // set to 1 when a bounded wait gave up
};

// 16 bytes of one row of a stage: EB = 4 -> 4 TF32 values, EB = 2 -> 8 BF16 values
template <int EB>
__device__ __forceinline__ uint4 load_unit(const float *row, int k0, int K, bool row_ok)
{
    uint4 v = make_uint4(0, 0, 0, 0);
    if (!row_ok) return v;
    if (EB == 4) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = (k0 + j < K) ? to_tf32(__ldg(row + k0 + j)) : 0u;
        v = make_uint4(w[0], w[1], w[2], w[3]);
    } else {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float a = (k0 + 2 * j < K) ? __ldg(row + k0 + 2 * j) : 0.f;
            const float c = (k0 + 2 * j + 1 < K) ? __ldg(row + k0 + 2 * j + 1) : 0.f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(a, c);
            w[j] = *reinterpret_cast<const uint32_t *>(&h);
        }
        v = make_uint4(w[0], w[1], w[2], w[3]);
    }
    return v;
}

// offset of (row r, 16-byte unit c) in a stage tile: 8-row groups 1024 bytes
// apart, units of one group 128 bytes apart, rows 16 bytes apart
__device__ __forceinline__ uint32_t tile_off(int r, int c)
{
    return (uint32_t)((r >> 3) * 1024 + c * 128 + (r & 7) * 16);
}

template <int EB>
__global__ void __launch_bounds__(kTcThreads, 1) tc_gemm_kernel(GemmParams<float> p, int BN)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base_sh;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int b_tile_bytes = BN * kChunk;
    const int stage_bytes = kATileBytes + b_tile_bytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int set = blockIdx.z;
    const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * BN;
    const float *A = p.A + set * p.strideA;
    const float *B = p.B + set * p.strideB;
    float *C = p.C + set * p.strideC;
    const uint32_t tcols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));

    if (warp == 0) {
        tmem_alloc(smem_addr(&tmem_base_sh), tcols);
        tmem_relinquish();
    }
    if (tid == 0) {
        mbar_init(smem_addr(&mbar[0]), 1);
        mbar_init(smem_addr(&mbar[1]), 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    constexpr int EPU = 16 / EB;                  // values per 16-byte unit
    constexpr int KC = kChunk / EB;               // values per stage row
    const int nchunks = (p.K + KC - 1) / KC;
    const uint32_t idesc = instr_desc(EB == 4 ? 2u : 1u, kTcBM, (uint32_t)BN);
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        const int s = c & 1;
        if (c >= 2) {
            bool w = ok ? mbar_wait(smem_addr(&mbar[s]), (uint32_t)((c - 2) >> 1) & 1u) : false;
            ok = __syncthreads_and(w) != 0;     // one decision for the whole block
        }
        uint8_t *sa = base + s * stage_bytes;
        uint8_t *sb = sa + kATileBytes;
        const int kbase = c * KC;
        for (int u = tid; u < kTcBM * 8; u += kTcThreads) {
            const int r = u >> 3, cu = u & 7;
            const int m = m0 + r;
            const uint4 v = load_unit<EB>(A + (int64_t)(m < p.M ? m : 0) * p.lda, kbase + cu * EPU, p.K, m < p.M);
            *reinterpret_cast<uint4 *>(sa + tile_off(r, cu)) = v;
        }
        for (int u = tid; u < BN * 8; u += kTcThreads) {
            const int r = u >> 3, cu = u & 7;
            const int n = n0 + r;
            const uint4 v = load_unit<EB>(B + (int64_t)(n < p.N ? n : 0) * p.ldb, kbase + cu * EPU, p.K, n < p.N);
            *reinterpret_cast<uint4 *>(sb + tile_off(r, cu)) = v;
        }
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && ok) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ad = smem_desc(smem_addr(sa) + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(smem_addr(sb) + ks * 256, 128, 1024);
                tc_mma<EB>(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            tc_commit(smem_addr(&mbar[s]));
        }
    }
    {
        bool w = ok ? mbar_wait(smem_addr(&mbar[(nchunks - 1) & 1]), (uint32_t)((nchunks - 1) >> 1) & 1u) : false;
        ok = __syncthreads_and(w) != 0;
    }
    tc_fence_after();
    float mx = 0.f;
    const int row = m0 + warp * 32 + lane;
    if (ok) {
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row < p.M) {
                float *dst = C + (int64_t)row * p.ldc + n0 + c0;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float v = __uint_as_float(r[j]);
                    if (n0 + c0 + j < p.N) {
                        dst[j] = v;
                        mx = fmaxf(mx, fabsf(v));
                    }
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(p.err, 1);
    }
    if (p.maxbits) {
        for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0 && mx > 0.f) atomicMax(p.maxbits + set, (unsigned long long)__float_as_uint(mx));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}

// FP64 on the CUDA cores: 64 x 64 tile, 16-deep K slab, 4 x 4 outputs per thread
constexpr int kF64Tile = 64, kF64Slab = 16;

__global__ void __launch_bounds__(256) f64_gemm_kernel(GemmParams<double> p)
{
    __shared__ double As[kF64Slab][kF64Tile + 1], Bs[kF64Slab][kF64Tile + 1];
    const int set = blockIdx.z;
    const int m0 = blockIdx.x * kF64Tile, n0 = blockIdx.y * kF64Tile;
    const double *A = p.A + set * p.strideA, *B = p.B + set * p.strideB;
    double *C = p.C + set * p.strideC;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < p.K; k0 += kF64Slab) {
        for (int i = threadIdx.x; i < kF64Slab * kF64Tile; i += blockDim.x) {
            const int r = i / kF64Slab, kk = i % kF64Slab;
            const int m = m0 + r, n = n0 + r, k = k0 + kk;
            As[kk][r] = (m < p.M && k < p.K) ? A[(int64_t)m * p.lda + k] : 0.0;
            Bs[kk][r] = (n < p.N && k < p.K) ? B[(int64_t)n * p.ldb + k] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kF64Slab; ++kk) {
            double a[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[kk][ty * 4 + i];
                bv[i] = Bs[kk][tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    double mx = 0.0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= p.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n < p.N) {
                C[(int64_t)m * p.ldc + n] = acc[i][j];
                mx = fmax(mx, fabs(acc[i][j]));
            }
        }
    }
    if (p.maxbits) {
        for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if ((threadIdx.x & 31) == 0 && mx > 0.0)
            atomicMax(p.maxbits + set, (unsigned long long)__double_as_longlong(mx));
    }
}

// ---------------------------------------------------------------- grid contraction
// A[m][u Kh + h] = 2^-e * S[u][m][h], e the exponent of the set's largest |S|
// (from maxbits[cur]); clears maxbits[next] and adds e to the set's log-2 scale.
template <typename T>
__global__ void grid_pack_kernel(const T *S, T *A, int64_t stride, int64_t R, int Ku, int Kh,
                                 unsigned long long *maxbits_cur, unsigned long long *maxbits_next,
                                 long long *log2s, int n_sets)
{
    const int set = blockIdx.y;
    if (set >= n_sets) return;
    const unsigned long long bits = maxbits_cur[set];
    int e = 0;
    if (sizeof(T) == 4) {
        const float mx = __uint_as_float((unsigned)bits);
        if (mx > 0.f) e = ilogbf(mx);
    } else {
        const double mx = __longlong_as_double((long long)bits);
        if (mx > 0.0) e = ilogb(mx);
    }
    const T sc = (T)ldexp(1.0, -e);
    const int K = Ku * Kh;
    const int64_t total = R * K;
    const T *s = S + set * stride;
    T *a = A + set * stride;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = q / K;
        const int k = (int)(q - m * K);
        const int u = k / Kh, h = k - u * Kh;
        a[q] = s[((int64_t)u * R + m) * Kh + h] * sc;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        maxbits_next[set] = 0ull;
        log2s[set] += e;
    }
}

// Site matrices B_v[n = d Nh + h'][k = u Kh + h] = 2^-s_v T_v[l = h, u, r = h', d]
// per (set, site): one block, the largest |entry| first (s_v its exponent).

template <typename T>
__global__ void grid_sites_kernel(const double *data, int64_t set_stride, const SiteMap *sites, int n_sites,
                                  T *Bm, int64_t b_stride, long long *log2s)
{
    const int v = blockIdx.x, set = blockIdx.y;
    const SiteMap sm = sites[v];
    const double *t = data + set * set_stride + sm.t_off;
    const int Kh = sm.dim[0], Ku = sm.dim[1], Nh = sm.dim[2], Nd = sm.dim[3];
    const int64_t n_ent = (int64_t)Kh * Ku * Nh * Nd;
    __shared__ double red[32];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n_ent; i += blockDim.x) mx = fmax(mx, fabs(t[i]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
        red[0] = mx;
    }
    __syncthreads();
    mx = red[0];
    const int e = mx > 0.0 ? ilogb(mx) : 0;
    const double sc = ldexp(1.0, -e);
    const int K = Ku * Kh, N = Nd * Nh;
    T *out = Bm + set * b_stride + sm.b_off;
    for (int64_t q = threadIdx.x; q < (int64_t)N * K; q += blockDim.x) {
        const int n = (int)(q / K), k = (int)(q % K);
        const int d = n / Nh, hp = n % Nh, u = k / Kh, h = k % Kh;
        const int64_t off = (int64_t)h * sm.stride[0] + (int64_t)u * sm.stride[1] + (int64_t)hp * sm.stride[2] +
                            (int64_t)d * sm.stride[3];
        out[q] = (T)(t[off] * sc);
    }
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long *>(log2s + set), (unsigned long long)(long long)e);
}

template <typename T>
__global__ void grid_init_kernel(T *S, int64_t stride, unsigned long long *maxbits, long long *log2s, int n_sets)
{
    const int set = blockIdx.x * blockDim.x + threadIdx.x;
    if (set >= n_sets) return;
    S[set * stride] = (T)1;
    maxbits[set] = sizeof(T) == 4 ? (unsigned long long)__float_as_uint(1.0f)
                                  : (unsigned long long)__double_as_longlong(1.0);
    log2s[set] = 0;
}

template <typename T>
__global__ void grid_final_kernel(const T *S, int64_t stride, const long long *log2s, int n_sets, double *out)
{
    const int set = blockIdx.x * blockDim.x + threadIdx.x;
    if (set >= n_sets) return;
    out[2 * set] = (double)S[set * stride];
    out[2 * set + 1] = (double)log2s[set];
}

// ---------------------------------------------------------------- the grid's pipelined GEMM
// One site absorption of the grid contraction on the tensor cores, with the
// running tensor S read in its ring order directly (no packing pass):
//     out[m][n] = 2^-e_in * sum_{u,h} S[u][m][h] * Bm[n][u Kh + h],
// the result rounded to the operand type (TF32 kept in FP32 words, or BF16) as
// the next step's running tensor, its largest |entry| recorded per set.
// Stages are filled with 16-byte cp.async copies (4 stages in flight): the
// operands are already in the MMA's type, so a stage is a plain copy into the
// canonical layout; where a 16-byte unit of A is not contiguous in S (a left
// boundary site, Kh not a multiple of the unit) it is gathered element by
// element instead.  The epilogue goes through shared memory (the free
// stages) so that every warp stores whole 128-byte row segments.
template <typename E>
struct RingParams {
    const E *S;              // [set][stride] running tensor [Ku][R][Kh]
    const E *B;              // site matrix [N][ldb] (rows zero-padded to ldb)
    E *out;                  // [set][stride] next running tensor [R][N]
    int64_t stride;          // running-tensor elements per set
    int64_t b_stride;        // site-matrix elements per set
    int64_t ldb;
    int64_t R;
    int Ku, Kh, N, K;
    const unsigned long long *max_in;   // [set] largest |S| (float bits)
    unsigned long long *max_out;        // [set] largest |out|, atomicMax
    unsigned long long *max_clear;      // [set] cleared for the next step
    long long *log2s;                   // [set] += e_in
    int *err;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

template <typename E>
__device__ __forceinline__ float elem_to_float(E x);
template <>
__device__ __forceinline__ float elem_to_float<float>(float x) { return x; }
template <>
__device__ __forceinline__ float elem_to_float<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

template <typename E>
__device__ __forceinline__ E round_elem(float x);
template <>
__device__ __forceinline__ float round_elem<float>(float x) { return __uint_as_float(to_tf32(x)); }
template <>
__device__ __forceinline__ __nv_bfloat16 round_elem<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

template <typename E, int NST>
__global__ void __launch_bounds__(kTcThreads, 2) tc_ring_gemm_kernel(RingParams<E> p, int BN)
{
    constexpr int kRingStages = NST;
    constexpr int EB = (int)sizeof(E);
    constexpr int EPU = 16 / EB;          // elements per 16-byte unit
    constexpr int KC = kChunk / EB;       // elements per stage row
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t mbar[kRingStages];
    __shared__ uint32_t tmem_base_sh;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int stage_bytes = kATileBytes + BN * kChunk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int set = blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * kTcBM;
    const int n0 = blockIdx.y * BN;
    const E *S = p.S + set * p.stride;
    const E *Bm = p.B + set * p.b_stride;
    E *out = p.out + set * p.stride;
    const uint32_t tcols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
    const bool a_contig = (p.Kh % EPU) == 0;

    if (warp == 0) {
        tmem_alloc(smem_addr(&tmem_base_sh), tcols);
        tmem_relinquish();
    }
    if (tid == 0)
        for (int i = 0; i < kRingStages; ++i) mbar_init(smem_addr(&mbar[i]), 1);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int nchunks = (p.K + KC - 1) / KC;
    const uint32_t idesc = instr_desc(EB == 4 ? 2u : 1u, kTcBM, (uint32_t)BN);

    // each thread copies one fixed 16-byte column (cu) of rows r0, r0 + 16, ...:
    // per stage one division for its k, then addresses advance by a constant
    const int cu = tid & 7, r0 = tid >> 3;
    const int64_t a_row_step = 16 * (int64_t)p.Kh;
    const int64_t b_row_step = 16 * p.ldb;
    auto load_stage = [&](int c) {
        if (c >= nchunks) return;
        uint8_t *sa = base + (c % kRingStages) * stage_bytes;
        uint8_t *sb = sa + kATileBytes;
        const int k = c * KC + cu * EPU;
        const bool k_in = k < p.K;
        if (a_contig) {
            const int ku = k_in ? k / p.Kh : 0, kh = k_in ? k - ku * p.Kh : 0;
            const E *src = S + ((int64_t)ku * p.R + m0 + r0) * p.Kh + kh;
            int64_t m = m0 + r0;
            uint32_t dst = smem_addr(sa) + (uint32_t)tile_off(r0, cu);
#pragma unroll
            for (int i = 0; i < kTcBM / 16; ++i) {
                const bool in = k_in && m < p.R;
                cp_async16(dst, in ? (const void *)src : (const void *)S, in ? 16u : 0u);
                src += a_row_step;
                m += 16;
                dst += 2 * 1024;            // 16 rows = two 8-row groups
            }
        } else {
            for (int i = 0; i < kTcBM / 16; ++i) {
                const int r = r0 + 16 * i;
                const int64_t m = m0 + r;
                __align__(16) E v[EPU];
#pragma unroll
                for (int j = 0; j < EPU; ++j) {
                    const int kk = k + j;
                    if (m < p.R && kk < p.K) {
                        const int ku = kk / p.Kh, kh = kk - ku * p.Kh;
                        v[j] = S[((int64_t)ku * p.R + m) * p.Kh + kh];
                    } else {
                        v[j] = round_elem<E>(0.f);
                    }
                }
                *reinterpret_cast<uint4 *>(sa + tile_off(r, cu)) = *reinterpret_cast<const uint4 *>(v);
            }
        }
        const uint32_t bytes = k_in ? (uint32_t)min(16, (p.K - k) * EB) : 0u;
        const E *bsrc = Bm + (int64_t)(n0 + r0) * p.ldb + (k_in ? k : 0);
        int n = n0 + r0;
        uint32_t bdst = smem_addr(sb) + (uint32_t)tile_off(r0, cu);
        for (int i = 0; i < BN / 16; ++i) {
            const bool in = n < p.N;
            cp_async16(bdst, in ? (const void *)bsrc : (const void *)Bm, in ? bytes : 0u);
            bsrc += b_row_step;
            n += 16;
            bdst += 2 * 1024;
        }
    };

    for (int c = 0; c < kRingStages - 1; ++c) {
        load_stage(c);
        cp_async_commit();
    }
    bool ok = true;
    for (int c = 0; c < nchunks; ++c) {
        cp_async_wait<kRingStages - 2>();
        fence_proxy_async();
        __syncthreads();
        if (tid == 0 && ok) {
            tc_fence_after();
            const uint8_t *sa = base + (c % kRingStages) * stage_bytes;
            const uint8_t *sb = sa + kATileBytes;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ad = smem_desc(smem_addr(sa) + ks * 256, 128, 1024);
                const uint64_t bd = smem_desc(smem_addr(sb) + ks * 256, 128, 1024);
                tc_mma<EB>(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            tc_commit(smem_addr(&mbar[c % kRingStages]));
        }
        // the stage the next prefetch overwrites was read by chunk c - 1
        if (c >= 1) {
            const bool w = ok ? mbar_wait(smem_addr(&mbar[(c - 1) % kRingStages]),
                                          (uint32_t)(((c - 1) / kRingStages) & 1))
                              : false;
            ok = __syncthreads_and(w) != 0;
        }
        load_stage(c + kRingStages - 1);
        cp_async_commit();
    }
    cp_async_wait<0>();
    {
        const int c = nchunks - 1;
        const bool w = ok ? mbar_wait(smem_addr(&mbar[c % kRingStages]), (uint32_t)((c / kRingStages) & 1)) : false;
        ok = __syncthreads_and(w) != 0;
    }
    tc_fence_after();
    // the scale of this step: 2^-e_in, e_in the exponent of the input's largest |entry|
    const float mx_in = __uint_as_float((unsigned)p.max_in[set]);
    const int e_in = mx_in > 0.f ? ilogbf(mx_in) : 0;
    const float sc = ldexpf(1.f, -e_in);
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        p.log2s[set] += e_in;
        p.max_clear[set] = 0ull;
    }
    float mx = 0.f;
    if (ok) {
        // 64-column slices through shared memory: [128][64 + 4] floats
        constexpr int SW = 64, SP = SW + 4;
        float *st = reinterpret_cast<float *>(base);
        for (int c0 = 0; c0 < BN; c0 += SW) {
#pragma unroll
            for (int q = 0; q < SW; q += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + q), r);
#pragma unroll
                for (int j = 0; j < 16; ++j) st[(warp * 32 + lane) * SP + q + j] = __uint_as_float(r[j]) * sc;
            }
            __syncthreads();
            for (int i = tid; i < kTcBM * SW; i += kTcThreads) {
                const int rr = i / SW, cc = i % SW;
                const int64_t row = m0 + rr;
                const int col = n0 + c0 + cc;
                if (row < p.R && col < p.N) {
                    const E v = round_elem<E>(st[rr * SP + cc]);
                    out[row * p.N + col] = v;
                    mx = fmaxf(mx, fabsf(elem_to_float<E>(v)));
                }
            }
            __syncthreads();
        }
    } else if (tid == 0) {
        atomicExch(p.err, 1);
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0 && mx > 0.f) atomicMax(p.max_out + set, (unsigned long long)__float_as_uint(mx));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
}

// Site matrices for the tensor-core path: rows padded to a multiple of the
// 16-byte unit, entries scaled by 2^-s_v and rounded to the operand type.
template <typename E>
__global__ void grid_sites_tc_kernel(const double *data, int64_t set_stride, const SiteMap *sites, E *Bm,
                                     int64_t b_stride, const int64_t *ldb, long long *log2s)
{
    const int v = blockIdx.x, set = blockIdx.y;
    const SiteMap sm = sites[v];
    const double *t = data + set * set_stride + sm.t_off;
    const int Kh = sm.dim[0], Ku = sm.dim[1], Nh = sm.dim[2], Nd = sm.dim[3];
    const int64_t n_ent = (int64_t)Kh * Ku * Nh * Nd;
    __shared__ double red[32];
    double mx = 0.0;
    for (int64_t i = threadIdx.x; i < n_ent; i += blockDim.x) mx = fmax(mx, fabs(t[i]));
    for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i) mx = fmax(mx, red[i]);
        red[0] = mx;
    }
    __syncthreads();
    mx = red[0];
    const int e = mx > 0.0 ? ilogb(mx) : 0;
    const double sc = ldexp(1.0, -e);
    const int K = Ku * Kh, N = Nd * Nh;
    const int64_t ld = ldb[v];
    E *out = Bm + set * b_stride + sm.b_off;
    for (int64_t q = threadIdx.x; q < (int64_t)N * ld; q += blockDim.x) {
        const int n = (int)(q / ld), k = (int)(q % ld);
        float x = 0.f;
        if (k < K) {
            const int d = n / Nh, hp = n % Nh, u = k / Kh, h = k % Kh;
            const int64_t off = (int64_t)h * sm.stride[0] + (int64_t)u * sm.stride[1] + (int64_t)hp * sm.stride[2] +
                                (int64_t)d * sm.stride[3];
            x = (float)(t[off] * sc);
        }
        out[q] = round_elem<E>(x);
    }
    if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long *>(log2s + set), (unsigned long long)(long long)e);
}

template <typename E>
__global__ void grid_init_tc_kernel(E *S, int64_t stride, unsigned long long *maxbits, long long *log2s, int n_sets)
{
    const int set = blockIdx.x * blockDim.x + threadIdx.x;
    if (set >= n_sets) return;
    S[set * stride] = round_elem<E>(1.f);
    maxbits[set] = (unsigned long long)__float_as_uint(1.0f);
    log2s[set] = 0;
}

template <typename E>
__global__ void grid_final_tc_kernel(const E *S, int64_t stride, const unsigned long long *max_last,
                                     const long long *log2s, int n_sets, double *out)
{
    const int set = blockIdx.x * blockDim.x + threadIdx.x;
    if (set >= n_sets) return;
    out[2 * set] = (double)elem_to_float<E>(S[set * stride]);
    out[2 * set + 1] = (double)log2s[set];
    (void)max_last;
}

// ---- the same site GEMM with the stages filled by the Tensor Memory Accelerator.
// One elected thread of warp 0 issues, per stage, eight boxes of A (the running
// tensor viewed as [set][Ku][R][Kh], each box 16 bytes of k by 128 rows) and
// eight of B ([set][N][ldb], 16 bytes of k by BN rows) on one mbarrier with
// the stage's byte count; a box lands as 128 (BN) consecutive 16-byte rows,
// which is the canonical no-swizzle K-major layout with 8-row groups 128
// bytes apart and the box's K column 2048 (16 BN) bytes from the next.  One
// thread of warp 1 waits for a full stage, issues its four MMAs and commits
// them to the stage's empty barrier, which the producer waits on before
// refilling it.  Used where a 16-byte unit of k is contiguous in the running
// tensor (Kh a multiple of the unit): the innermost box coordinate is then a
// multiple of 16 bytes, as the copy requires.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                          uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], [%6];"
                 ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, uint32_t bar)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
                 ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tma_load3_mc(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                             uint32_t bar, uint16_t mask)
{
    asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster"
                 " [%0], [%1, {%2, %3, %4}], [%5], %6;"
                 ::"r"(dst), "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(c2), "r"(bar), "h"(mask)
                 : "memory");
}
__device__ __forceinline__ void tc_commit_mc(uint32_t mbar, uint16_t mask)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;"
                 ::"r"(mbar), "h"(mask)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// CL CTAs on adjacent M tiles form a cluster and share the site matrix: each
// loads 1/CL of every stage's B boxes and multicasts them to all, so the L2
// delivers B once per cluster instead of once per CTA.  A stage is refilled
// only after every member's MMAs on it completed (each member's commit
// arrives on every member's empty barrier, CL arrivals per phase).
template <typename E, int NST, int CL>
__global__ void __launch_bounds__(kTcThreads, 2) tc_tma_gemm_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB,
                                                                   RingParams<E> p, int BN)
{
    constexpr int EB = (int)sizeof(E);
    constexpr int EPU = 16 / EB;
    constexpr int KC = kTmaChunk / EB;        // k values per stage (64 bytes of each row)
    constexpr int UNITS = kTmaChunk / 16;     // 16-byte boxes per operand per stage
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[NST], empty[NST], done;
    __shared__ uint32_t tmem_base_sh;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int a_bytes = kTcBM * kTmaChunk;
    const int stage_bytes = a_bytes + BN * kTmaChunk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int set = blockIdx.z;
    const int64_t m0 = (int64_t)blockIdx.x * kTcBM;
    const int n0 = blockIdx.y * BN;
    E *out = p.out + set * p.stride;
    const uint32_t tcols = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u));
    uint32_t crank = 0;
    if (CL > 1) asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(crank));
    const uint16_t cmask = (uint16_t)((1u << CL) - 1u);
    if (warp == 0) {
        tmem_alloc(smem_addr(&tmem_base_sh), tcols);
        tmem_relinquish();
    }
    if (tid == 32) {
        for (int i = 0; i < NST; ++i) {
            mbar_init(smem_addr(&full[i]), 1);
            mbar_init(smem_addr(&empty[i]), CL);
        }
        mbar_init(smem_addr(&done), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    if (CL > 1) cluster_sync_all();      // every member's barriers exist before any multicast
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int nchunks = (p.K + KC - 1) / KC;
    const uint32_t idesc = instr_desc(EB == 4 ? 2u : 1u, kTcBM, (uint32_t)BN);
    const uint32_t stage_tx = (uint32_t)stage_bytes;
    int failed = 0;
    if (tid == 0) {
        // producer
        for (int c = 0; c < nchunks && !failed; ++c) {
            const int s = c % NST;
            if (c >= NST && !mbar_wait(smem_addr(&empty[s]), (uint32_t)(((c / NST) - 1) & 1))) {
                failed = 1;
                break;
            }
            const uint32_t fb = smem_addr(&full[s]);
            mbar_expect_tx(fb, stage_tx);
            const uint32_t sa = smem_addr(base + s * stage_bytes), sb = sa + a_bytes;
#pragma unroll
            for (int cu = 0; cu < UNITS; ++cu) {
                const int k = c * KC + cu * EPU;
                const int ku = k / p.Kh, kh = k - ku * p.Kh;
                tma_load4(sa + cu * (kTcBM * 16), &tmA, kh, (int)m0, ku, set, fb);
                if (CL == 1)
                    tma_load3(sb + cu * (BN * 16), &tmB, k, n0, set, fb);
                else if (cu % CL == (int)crank)
                    tma_load3_mc(sb + cu * (BN * 16), &tmB, k, n0, set, fb, cmask);
            }
        }
    } else if (tid == 32) {
        // MMA issuer
        for (int c = 0; c < nchunks; ++c) {
            const int s = c % NST;
            if (!mbar_wait(smem_addr(&full[s]), (uint32_t)((c / NST) & 1))) {
                failed = 1;
                break;
            }
            tc_fence_after();
            const uint32_t sa = smem_addr(base + s * stage_bytes), sb = sa + a_bytes;
#pragma unroll
            for (int ks = 0; ks < UNITS / 2; ++ks) {
                const uint64_t ad = smem_desc(sa + ks * 2 * (kTcBM * 16), kTcBM * 16, 128);
                const uint64_t bd = smem_desc(sb + ks * 2 * (BN * 16), (uint32_t)(BN * 16), 128);
                tc_mma<EB>(tmem, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
            }
            if (CL == 1) tc_commit(smem_addr(&empty[s]));
            else tc_commit_mc(smem_addr(&empty[s]), cmask);
        }
        if (!failed) tc_commit(smem_addr(&done));
    }
    // everyone: the accumulator is complete once `done` fires
    bool ok = __syncthreads_or(failed) == 0;
    if (ok) ok = mbar_wait(smem_addr(&done), 0u);
    ok = __syncthreads_and(ok) != 0;
    tc_fence_after();
    const float mx_in = __uint_as_float((unsigned)p.max_in[set]);
    const int e_in = mx_in > 0.f ? ilogbf(mx_in) : 0;
    const float sc = ldexpf(1.f, -e_in);
    if (blockIdx.x == 0 && blockIdx.y == 0 && tid == 0) {
        p.log2s[set] += e_in;
        p.max_clear[set] = 0ull;
    }
    float mx = 0.f;
    if (ok) {
        constexpr int SW = 64, SP = SW + 4;
        float *st = reinterpret_cast<float *>(base);
        for (int c0 = 0; c0 < BN; c0 += SW) {
#pragma unroll
            for (int q = 0; q < SW; q += 16) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c0 + q), r);
#pragma unroll
                for (int j = 0; j < 16; ++j) st[(warp * 32 + lane) * SP + q + j] = __uint_as_float(r[j]) * sc;
            }
            __syncthreads();
            for (int i = tid; i < kTcBM * SW; i += kTcThreads) {
                const int rr = i / SW, cc = i % SW;
                const int64_t row = m0 + rr;
                const int col = n0 + c0 + cc;
                if (row < p.R && col < p.N) {
                    const E v = round_elem<E>(st[rr * SP + cc]);
                    out[row * p.N + col] = v;
                    mx = fmaxf(mx, fabsf(elem_to_float<E>(v)));
                }
            }
            __syncthreads();
        }
    } else if (tid == 0) {
        atomicExch(p.err, 1);
    }
    for (int off = 16; off > 0; off >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
    if (lane == 0 && mx > 0.f) atomicMax(p.max_out + set, (unsigned long long)__float_as_uint(mx));
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, tcols);
    if (CL > 1) cluster_sync_all();      // no member leaves while another may still signal it
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    });
    return fn;
}

template <typename E, int NST, int CL>
cudaError_t launch_tma_n(const RingParams<E> &p, int batch, int BN, int n_sets, cudaStream_t s, bool &used)
{
    used = false;
    auto enc = tensor_map_encoder();
    if (!enc) return cudaSuccess;
    constexpr int EB = (int)sizeof(E);
    const CUtensorMapDataType dt = EB == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    CUtensorMap ma, mb;
    // A: [set][Ku][R][Kh], innermost first
    const cuuint64_t adim[4] = {(cuuint64_t)p.Kh, (cuuint64_t)p.R, (cuuint64_t)p.Ku, (cuuint64_t)n_sets};
    const cuuint64_t astr[3] = {(cuuint64_t)p.Kh * EB, (cuuint64_t)p.R * p.Kh * EB, (cuuint64_t)p.stride * EB};
    const cuuint32_t abox[4] = {(cuuint32_t)(16 / EB), (cuuint32_t)kTcBM, 1, 1};
    const cuuint32_t one4[4] = {1, 1, 1, 1};
    // B: [set][N][ldb]
    const cuuint64_t bdim[3] = {(cuuint64_t)p.ldb, (cuuint64_t)p.N, (cuuint64_t)n_sets};
    const cuuint64_t bstr[2] = {(cuuint64_t)p.ldb * EB, (cuuint64_t)p.b_stride * EB};
    const cuuint32_t bbox[3] = {(cuuint32_t)(16 / EB), (cuuint32_t)BN, 1};
    if (enc(&ma, dt, 4, (void *)p.S, adim, astr, abox, one4, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS ||
        enc(&mb, dt, 3, (void *)p.B, bdim, bstr, bbox, one4, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) !=
            CUDA_SUCCESS)
        return cudaSuccess;         // not encodable: the copy-loop kernel runs instead
    // the epilogue stages the accumulator through the same shared memory: 128 x 68 floats
    const size_t smem = std::max<size_t>((size_t)NST * (kTcBM + BN) * kTmaChunk, (size_t)kTcBM * 68 * 4) + 1024;
    cudaError_t e = grant_dynamic_smem((const void *)tc_tma_gemm_kernel<E, NST, CL>, smem);
    if (e != cudaSuccess) return e;
    const int64_t mt = (p.R + kTcBM - 1) / kTcBM;
    const dim3 grid((unsigned)((mt + CL - 1) / CL * CL), (unsigned)((p.N + BN - 1) / BN), (unsigned)batch);
    if (CL == 1) {
        tc_tma_gemm_kernel<E, NST, CL><<<grid, kTcThreads, smem, s>>>(ma, mb, p, BN);
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = dim3(kTcThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = CL;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, tc_tma_gemm_kernel<E, NST, CL>, ma, mb, p, BN);
        if (e != cudaSuccess) return e;
    }
    used = true;
    return cudaGetLastError();
}

// stages per CTA: as many as let two CTAs share an SM (<= 113 KB each, 2 x 256
// tensor-memory columns), so one CTA's prologue and epilogue overlap the
// other's main loop
template <typename E, int NST>
cudaError_t launch_ring_n(const RingParams<E> &p, int batch, int BN, cudaStream_t s)
{
    const size_t smem = (size_t)NST * (kATileBytes + BN * kChunk) + 1024;
    cudaError_t e = grant_dynamic_smem((const void *)tc_ring_gemm_kernel<E, NST>, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((p.R + kTcBM - 1) / kTcBM), (unsigned)((p.N + BN - 1) / BN), (unsigned)batch);
    tc_ring_gemm_kernel<E, NST><<<grid, kTcThreads, smem, s>>>(p, BN);
    return cudaGetLastError();
}

template <typename E>
cudaError_t launch_ring(const RingParams<E> &p, int batch, cudaStream_t s)
{
    const int BN = std::min(256, ((p.N + 15) / 16) * 16);
    const int stage = kATileBytes + BN * kChunk;
    const int nst = (int)std::max<int64_t>(2, std::min<int64_t>(4, (112 * 1024) / stage));
    constexpr int EPU = 16 / (int)sizeof(E);
    // TMA where every 16-byte unit of k is contiguous and every stride a multiple of 16 bytes
    if (p.Kh % EPU == 0 && (p.ldb % EPU) == 0 && (p.stride % EPU) == 0 && (p.b_stride % EPU) == 0 &&
        p.R < (int64_t)1 << 31) {
        bool used = false;
        // 64-byte stages: twice as many in flight in the same shared memory (two CTAs per SM)
        const int tstage = (kTcBM + BN) * kTmaChunk;
        const int tn = (int)std::max<int64_t>(2, std::min<int64_t>(8, (112 * 1024) / tstage));
        // clusters of CL CTAs share the site matrix through multicast (PNE_TC_CLUSTER = 1, 2 or 4;
        // default 2) when the rows fill at least two clusters
        static const int cl_env = [] {
            const char *v = std::getenv("PNE_TC_CLUSTER");
            const int c = v ? std::atoi(v) : 2;
            return (c == 1 || c == 2 || c == 4) ? c : 2;
        }();
        const int64_t mt = (p.R + kTcBM - 1) / kTcBM;
        const int cl = mt >= 2 * cl_env ? cl_env : 1;
        cudaError_t e;
        if (cl == 4)
            e = tn >= 8 ? launch_tma_n<E, 8, 4>(p, batch, BN, batch, s, used) : launch_tma_n<E, 4, 4>(p, batch, BN, batch, s, used);
        else if (cl == 2)
            e = tn >= 8 ? launch_tma_n<E, 8, 2>(p, batch, BN, batch, s, used) : launch_tma_n<E, 4, 2>(p, batch, BN, batch, s, used);
        else
            e = tn >= 8   ? launch_tma_n<E, 8, 1>(p, batch, BN, batch, s, used)
                : tn >= 4 ? launch_tma_n<E, 4, 1>(p, batch, BN, batch, s, used)
                          : launch_tma_n<E, 2, 1>(p, batch, BN, batch, s, used);
        if (e != cudaSuccess || used) return e;
    }
    if (nst >= 4) return launch_ring_n<E, 4>(p, batch, BN, s);
    if (nst == 3) return launch_ring_n<E, 3>(p, batch, BN, s);
    return launch_ring_n<E, 2>(p, batch, BN, s);
}

size_t tc_smem_bytes(int BN)
{
    return (size_t)2 * (kATileBytes + BN * kChunk) + 1024;
}

template <int EB>
cudaError_t launch_tc(const GemmParams<float> &p, int batch, cudaStream_t s)
{
    const int BN = std::min(256, ((p.N + 15) / 16) * 16);
    const size_t smem = tc_smem_bytes(BN);
    cudaError_t e = grant_dynamic_smem((const void *)tc_gemm_kernel<EB>, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((p.M + kTcBM - 1) / kTcBM), (unsigned)((p.N + BN - 1) / BN), (unsigned)batch);
    tc_gemm_kernel<EB><<<grid, kTcThreads, smem, s>>>(p, BN);
    return cudaGetLastError();
}

cudaError_t launch_f64(const GemmParams<double> &p, int batch, cudaStream_t s)
{
    const dim3 grid((unsigned)((p.M + kF64Tile - 1) / kF64Tile), (unsigned)((p.N + kF64Tile - 1) / kF64Tile),
                    (unsigned)batch);
    f64_gemm_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace

pne_status grid_plan(pne_ctx *ctx, int lx, int ly, int n_bonds, const int32_t *bond_site, const int32_t *bond_dim,
                     const int32_t *site_ptr, const int32_t *site_bonds, const int64_t *data_off, pne_dtype dtype,
                     int nb, GridPlan &plan)
{
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    const int n = lx * ly;
    // bond between grid neighbours: horizontal hb[v] (x, y)-(x+1, y), vertical vb[v] (x, y)-(x, y+1)
    std::vector<int> hb((size_t)n, -1), vb((size_t)n, -1);
    for (int b = 0; b < n_bonds; ++b) {
        int s0 = bond_site[2 * b], s1 = bond_site[2 * b + 1];
        if (s0 < 0 || s1 < 0 || s0 >= n || s1 >= n) return bad("grid networks have no open indices");
        if (s0 > s1) std::swap(s0, s1);
        const int x0 = s0 % lx, y0 = s0 / lx, x1 = s1 % lx, y1 = s1 / lx;
        const int d = bond_dim[b];
        if (d < 1 || d > 4096) return bad("bond dimension out of range");
        if (y0 == y1 && x1 == x0 + 1) {
            if (hb[s0] >= 0) return bad("two bonds join the same grid neighbours");
            hb[s0] = b;
        } else if (x0 == x1 && y1 == y0 + 1) {
            if (vb[s0] >= 0) return bad("two bonds join the same grid neighbours");
            vb[s0] = b;
        } else {
            return bad("a bond does not join grid neighbours (site id = y * lx + x)");
        }
    }
    for (int y = 0; y < ly; ++y)
        for (int x = 0; x < lx; ++x) {
            const int v = y * lx + x;
            if ((x + 1 < lx && hb[v] < 0) || (y + 1 < ly && vb[v] < 0)) return bad("a grid bond is missing");
        }
    plan.n = n;
    plan.maps.assign((size_t)n, SiteMap{});
    plan.steps.assign((size_t)n, GridStep{});
    plan.ldb.assign((size_t)n, 0);
    const size_t esz = dtype == PNE_F64 ? 8 : (dtype == PNE_TF32 ? 4 : 2);
    const int epu = dtype == PNE_F64 ? 1 : (int)(16 / esz);
    int64_t b_total = 0, state = 1, max_state = 1;
    for (int y = 0; y < ly; ++y)
        for (int x = 0; x < lx; ++x) {
            const int v = y * lx + x;
            const int legb[4] = {x > 0 ? hb[v - 1] : -1, y > 0 ? vb[v - lx] : -1, x + 1 < lx ? hb[v] : -1,
                                 y + 1 < ly ? vb[v] : -1};
            SiteMap &sm = plan.maps[(size_t)v];
            const int p0 = site_ptr[v], p1 = site_ptr[v + 1];
            int nlegs = 0;
            for (int i = 0; i < 4; ++i) nlegs += legb[i] >= 0;
            if (p1 - p0 != nlegs) return bad("a site's legs are not its grid bonds");
            for (int i = 0; i < 4; ++i) {
                sm.dim[i] = legb[i] >= 0 ? bond_dim[legb[i]] : 1;
                sm.stride[i] = 0;
            }
            // strides: legs in the order of site_bonds, row-major
            int64_t stride = 1;
            for (int q = p1 - 1; q >= p0; --q) {
                const int b = site_bonds[q];
                int which = -1;
                for (int i = 0; i < 4; ++i)
                    if (legb[i] == b) which = i;
                if (which < 0) return bad("a site's legs are not its grid bonds");
                if (stride > INT32_MAX) return bad("site tensor too large");
                sm.stride[which] = (int)stride;
                stride *= bond_dim[b];
            }
            if (data_off[v + 1] - data_off[v] != stride) return bad("data_off does not match the bond dims");
            sm.t_off = data_off[v];
            GridStep sd{sm.dim[1], sm.dim[0], sm.dim[3], sm.dim[2], 0};
            const int64_t K = (int64_t)sd.Ku * sd.Kh;
            if (state % K != 0) return bad("internal: running tensor does not split");
            sd.R = state / K;
            if (sd.R > INT32_MAX || (int64_t)sd.Nd * sd.Nh > INT32_MAX || K > INT32_MAX)
                return bad("a step's matrix is too large");
            plan.ldb[(size_t)v] = (K + epu - 1) / epu * epu;
            sm.b_off = b_total;
            b_total += plan.ldb[(size_t)v] * sd.Nd * sd.Nh;
            state = sd.R * sd.Nd * sd.Nh;
            max_state = std::max(max_state, std::max(state, sd.R * K));
            plan.steps[(size_t)v] = sd;
        }
    if (state != 1) return bad("internal: the contraction did not close");
    plan.b_total = b_total;
    plan.max_state = (max_state + 63) / 64 * 64;
    if ((double)plan.max_state * esz * 2 * nb > 64e9) return bad("running tensors exceed 64 GB for this batch");
    return PNE_OK;
}

pne_status grid_run(pne_ctx *ctx, const GridPlan &plan, const double *data, int64_t set_stride, int nb,
                    pne_dtype dtype, cudaStream_t s, std::vector<double> &h, double &bound)
{
    const int n = plan.n;
    const size_t esz = dtype == PNE_F64 ? 8 : (dtype == PNE_TF32 ? 4 : 2);
    const int64_t max_state = plan.max_state, b_total = plan.b_total;
    DevBuf dMaps, dB, dS, dA, dMax, dLog, dOut, dErr, dLdb;
    auto cleanup = [&]() {
        for (DevBuf *b : {&dMaps, &dB, &dS, &dA, &dMax, &dLog, &dOut, &dErr, &dLdb}) dev_free(ctx, *b, s);
    };
    pne_status st;
    if ((st = dev_alloc(ctx, dMaps, plan.maps.size() * sizeof(SiteMap), s)) ||
        (st = dev_alloc(ctx, dB, (size_t)nb * b_total * esz, s)) ||
        (st = dev_alloc(ctx, dS, (size_t)nb * max_state * esz, s)) ||
        (st = dev_alloc(ctx, dA, (size_t)nb * max_state * esz, s)) || (st = dev_alloc(ctx, dMax, (size_t)nb * 24, s)) ||
        (st = dev_alloc(ctx, dLog, (size_t)nb * 8, s)) || (st = dev_alloc(ctx, dOut, (size_t)nb * 16, s)) ||
        (st = dev_alloc(ctx, dErr, 16, s)) || (st = dev_alloc(ctx, dLdb, (size_t)n * 8, s))) {
        cleanup();
        return st;
    }
    auto fail = [&](cudaError_t e, const char *what) {
        set_error(ctx, PNE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
        cleanup();
        return PNE_ECUDA;
    };
    cudaError_t e = cudaMemcpyAsync(dMaps.ptr, plan.maps.data(), plan.maps.size() * sizeof(SiteMap),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dLdb.ptr, plan.ldb.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dErr.ptr, 0, 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dMax.ptr, 0, (size_t)nb * 24, s);
    if (e != cudaSuccess) return fail(e, "grid upload");
    unsigned long long *mb = (unsigned long long *)dMax.ptr;
    long long *lg = (long long *)dLog.ptr;
    const int ib = (nb + 127) / 128;
    bound = 0.0;
    const double u_in = dtype == PNE_TF32 ? std::ldexp(1.0, -11) : (dtype == PNE_BF16 ? std::ldexp(1.0, -8) : 0.0);
    if (dtype != PNE_F64) {
        // running tensors ping-pong between dS and dA; largest |entry| in three rotating slots
        auto run_tc = [&](auto tag) -> cudaError_t {
            using E = decltype(tag);
            E *S0 = (E *)dS.ptr, *S1 = (E *)dA.ptr;
            {
                ProfScope ps(ctx, s, "grid_sites");
                grid_init_tc_kernel<E><<<ib, 128, 0, s>>>(S0, max_state, mb, lg, nb);
                grid_sites_tc_kernel<E><<<dim3(n, nb), 256, 0, s>>>(data, set_stride, (const SiteMap *)dMaps.ptr,
                                                                    (E *)dB.ptr, b_total, (const int64_t *)dLdb.ptr, lg);
            }
            cudaError_t ee = cudaGetLastError();
            if (ee != cudaSuccess) return ee;
            for (int v = 0; v < n; ++v) {
                const GridStep &sd = plan.steps[(size_t)v];
                RingParams<E> rp;
                rp.S = (v & 1) ? S1 : S0;
                rp.out = (v & 1) ? S0 : S1;
                rp.B = (const E *)dB.ptr + plan.maps[(size_t)v].b_off;
                rp.stride = max_state;
                rp.b_stride = b_total;
                rp.ldb = plan.ldb[(size_t)v];
                rp.R = sd.R;
                rp.Ku = sd.Ku;
                rp.Kh = sd.Kh;
                rp.N = sd.Nd * sd.Nh;
                rp.K = sd.Ku * sd.Kh;
                rp.max_in = mb + (size_t)(v % 3) * nb;
                rp.max_out = mb + (size_t)((v + 1) % 3) * nb;
                rp.max_clear = mb + (size_t)((v + 2) % 3) * nb;
                rp.log2s = lg;
                rp.err = (int *)dErr.ptr;
                ProfScope ps(ctx, s, "grid_gemm_tc");
                if ((ee = launch_ring<E>(rp, nb, s)) != cudaSuccess) return ee;
                bound += 2.0 * u_in + (double)rp.K * std::ldexp(1.0, -24);
            }
            {
                ProfScope ps(ctx, s, "grid_final");
                grid_final_tc_kernel<E><<<ib, 128, 0, s>>>((n & 1) ? S1 : S0, max_state, mb, lg, nb, (double *)dOut.ptr);
            }
            return cudaGetLastError();
        };
        e = dtype == PNE_TF32 ? run_tc(float(0)) : run_tc(__nv_bfloat16());
        if (e != cudaSuccess) return fail(e, "grid contraction (tensor cores)");
    } else {
        {
            ProfScope ps(ctx, s, "grid_sites");
            grid_init_kernel<double><<<ib, 128, 0, s>>>((double *)dS.ptr, max_state, mb, lg, nb);
            grid_sites_kernel<double><<<dim3(n, nb), 256, 0, s>>>(data, set_stride, (const SiteMap *)dMaps.ptr, n,
                                                                  (double *)dB.ptr, b_total, lg);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "grid site matrices");
        for (int v = 0; v < n; ++v) {
            const GridStep &sd = plan.steps[(size_t)v];
            const int K = sd.Ku * sd.Kh, N = sd.Nd * sd.Nh;
            unsigned long long *cur = mb + (size_t)(v & 1) * nb, *nxt = mb + (size_t)((v + 1) & 1) * nb;
            const int64_t total = sd.R * K;
            const int pblocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 8);
            {
                ProfScope ps(ctx, s, "grid_pack");
                grid_pack_kernel<double><<<dim3(pblocks, nb), 256, 0, s>>>((const double *)dS.ptr, (double *)dA.ptr,
                                                                          max_state, sd.R, sd.Ku, sd.Kh, cur, nxt, lg,
                                                                          nb);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "grid_pack_kernel");
            {
                ProfScope ps(ctx, s, "grid_gemm_f64");
                GemmParams<double> p{(const double *)dA.ptr, K, max_state,
                                     (const double *)dB.ptr + plan.maps[(size_t)v].b_off, K, b_total,
                                     (double *)dS.ptr, N, max_state, (int)sd.R, N, K, nxt, (int *)dErr.ptr};
                e = launch_f64(p, nb, s);
            }
            if (e != cudaSuccess) return fail(e, "grid GEMM");
            bound += (double)K * std::ldexp(1.0, -53);
        }
        {
            ProfScope ps(ctx, s, "grid_final");
            grid_final_kernel<double><<<ib, 128, 0, s>>>((const double *)dS.ptr, max_state, lg, nb, (double *)dOut.ptr);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "grid_final_kernel");
    }
    h.assign((size_t)nb * 2, 0.0);
    int herr = 0;
    if ((e = cudaMemcpyAsync(h.data(), dOut.ptr, h.size() * 8, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&herr, dErr.ptr, 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(e, "grid results");
    cleanup();
    if (herr) {
        set_error(ctx, PNE_ETIMEOUT, "grid contraction: a tensor-core stage wait gave up");
        return PNE_ETIMEOUT;
    }
    return PNE_OK;
}

}  // namespace pne

using namespace pne;

extern "C" {

pne_status pne_dense_gemm(pne_ctx *ctx, pne_dtype dtype, int32_t batch, int32_t M, int32_t N, int32_t K,
                          const void *A, int64_t lda, int64_t strideA, const void *B, int64_t ldb, int64_t strideB,
                          void *C, int64_t ldc, int64_t strideC, void *stream)
{
    HostScope hs__(ctx, "dense_gemm");
    if (!ctx || !A || !B || !C) return PNE_EINVAL;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    if (batch < 1 || batch > 65535 || M < 1 || N < 1 || K < 1) return bad("batch in 1..65535, M, N, K >= 1");
    if (lda < K || ldb < K || ldc < N) return bad("leading dimensions below K (A, B) or N (C)");
    if (dtype == PNE_F32) return bad("dense_gemm takes PNE_F64, PNE_TF32 or PNE_BF16");
    cudaStream_t s = (cudaStream_t)stream;
    DevBuf err;
    pne_status st = dev_alloc(ctx, err, 16, s);
    if (st) return st;
    cudaError_t e = cudaMemsetAsync(err.ptr, 0, 16, s);
    if (e == cudaSuccess) {
        ProfScope ps(ctx, s, dtype == PNE_F64 ? "dense_gemm_f64" : "dense_gemm_tc");
        if (dtype == PNE_F64) {
            GemmParams<double> p{(const double *)A, lda, strideA, (const double *)B, ldb, strideB, (double *)C, ldc,
                                 strideC, M, N, K, nullptr, (int *)err.ptr};
            e = launch_f64(p, batch, s);
        } else {
            GemmParams<float> p{(const float *)A, lda, strideA, (const float *)B, ldb, strideB, (float *)C, ldc,
                                strideC, M, N, K, nullptr, (int *)err.ptr};
            e = dtype == PNE_TF32 ? launch_tc<4>(p, batch, s) : launch_tc<2>(p, batch, s);
        }
    }
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err.ptr, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(ctx, err, s);
    if (e != cudaSuccess) {
        set_error(ctx, PNE_ECUDA, std::string("dense_gemm: ") + cudaGetErrorString(e));
        return PNE_ECUDA;
    }
    if (herr) {
        set_error(ctx, PNE_ETIMEOUT, "dense_gemm: a tensor-core stage wait gave up");
        return PNE_ETIMEOUT;
    }
    return PNE_OK;
}

pne_status pne_grid_contract(pne_ctx *ctx, const pne_network *net, int32_t lx, int32_t ly, pne_dtype dtype,
                             void *stream, pne_result *out)
{
    HostScope hs__(ctx, "grid_contract");
    if (!ctx || !net || !out) return PNE_EINVAL;
    auto bad = [&](const std::string &m) { set_error(ctx, PNE_EINVAL, m); return PNE_EINVAL; };
    if (dtype == PNE_F32) return bad("grid_contract takes PNE_F64, PNE_TF32 or PNE_BF16");
    const int nb = net->n_batch;
    if (nb < 1 || nb > 65535) return bad("n_batch in 1..65535");
    if (!net->bond_site || !net->bond_dim || !net->site_ptr || !net->site_bonds || !net->data || !net->data_off)
        return bad("null network array");
    if (lx < 1 || ly < 1 || (int64_t)lx * ly != net->n_sites) return bad("n_sites must be lx * ly");
    GridPlan plan;
    pne_status st = grid_plan(ctx, lx, ly, net->n_bonds, net->bond_site, net->bond_dim, net->site_ptr,
                              net->site_bonds, net->data_off, dtype, nb, plan);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t set_stride = net->data_off[net->n_sites];
    DevBuf dData;
    const double *data = net->data;
    if (!net->data_on_device) {
        if ((st = dev_alloc(ctx, dData, (size_t)nb * set_stride * 8, s))) return st;
        if ((st = upload(ctx, dData.ptr, net->data, (size_t)nb * set_stride * 8, s))) {
            dev_free(ctx, dData, s);
            return st;
        }
        data = (const double *)dData.ptr;
    }
    std::vector<double> h;
    double bound = 0.0;
    st = grid_run(ctx, plan, data, set_stride, nb, dtype, s, h, bound);
    dev_free(ctx, dData, s);
    if (st != PNE_OK && st != PNE_ETIMEOUT) return st;
    for (int b = 0; b < nb; ++b) {
        pne_result &r = out[b];
        std::memset(&r, 0, sizeof(r));
        const double m = h[2 * b], l2 = h[2 * b + 1];
        r.sign = m > 0 ? 1 : (m < 0 ? -1 : 0);
        r.log_abs = m != 0 ? std::log(std::fabs(m)) + l2 * std::log(2.0) : -INFINITY;
        r.value = m != 0 ? (double)r.sign * std::exp(r.log_abs) : 0.0;
        r.n_orders = 1;
        r.c[0] = 1.0;
        r.abs_c[0] = 1.0;
        r.log_abs_zref = r.log_abs;
        r.sign_zref = r.sign;
        r.log_series = r.log_abs;
        r.err_bound = bound;
        r.n_terms = 1;
    }
    return st;
}

}  // extern "C"
