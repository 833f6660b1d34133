// Resistance-tensor surrogate: tensor-core GEMM (tcgen05), the network's
// loss / backward / Adam kernels and small SPD solves, behind
// include/lbsurrogate.h.
//
// GEMM (C = A B^T, BF16 operands, FP32 accumulation): one CTA of one
// warpgroup (128 threads) per 128 x N tile (N <= 256).  For each K chunk of 64
// the threads stage A (128 x 64) and B (N x 64) into shared memory in the
// canonical no-swizzle K-major layout of 8-row x 16-byte core matrices (core
// (g, c) of rows 8g.. and K columns 8c.. at byte (8g + c) * 128, so adjacent
// core matrices are 128 bytes apart along K and 1024 bytes apart along the
// rows); one elected thread issues four tcgen05.mma (M = 128, K = 16 each)
// accumulating in tensor memory and commits them to an mbarrier that every
// thread waits on (bounded).  Two stages: while the products of chunk c run,
// the threads stage chunk c + 1 into the other stage (whose products, those of
// chunk c - 1, were waited for).  The staging loads are coalesced for either
// operand layout: 16-byte loads of 8 consecutive K (K-major operands) or of 8
// consecutive rows (transposed operands) where strides and alignment allow,
// else one element per thread with consecutive threads on the contiguous
// index.  The
// epilogue: warp w reads TMEM lanes 32w..32w+31 (one output row per lane) with
// tcgen05.ld, adds the bias, applies ReLU and writes FP32 and/or BF16.
// The network is small (8 -> 256 -> 256 -> 21), so the staging is done by
// plain loads that also transpose; the products are the only dense
// contractions and the only work on the tensor cores.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/lbsurrogate.h"

namespace lbsur {

constexpr int GM = 128;                 // tile rows: one TMEM lane per row
constexpr int GN = 256;                 // widest tile (one MMA, N <= 256)
constexpr int GK = 64;                  // K chunk per staging round
constexpr int GTHREADS = 128;           // one warpgroup
constexpr int SMEM_A = GM * GK * 2;     // 16 KiB
constexpr int SMEM_B = GN * GK * 2;     // 32 KiB
constexpr int GEMM_STAGE = SMEM_A + SMEM_B;
constexpr int GEMM_SMEM = 2 * GEMM_STAGE; // two stages, 96 KiB
constexpr long long SPIN_LIMIT = 1ll << 24;

struct GemmArgs {
    const __nv_bfloat16* A;
    long long a_sm, a_sk;
    const __nv_bfloat16* B;
    long long b_sn, b_sk;
    int M, N, K;
    const float* bias;
    int relu;
    const __nv_bfloat16* mask;          // if set: C *= (mask(m, n) > 0), same strides as C
    float* C32;
    __nv_bfloat16* C16;
    long long c_sm, c_sn;
    unsigned* status;
};

__device__ unsigned g_gemm_status;      // bit 0: a completion wait gave up

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-major, byte offsets between
// core matrices along K (lbo) and along the rows (sbo); bits 46-48 = 0b001
__device__ __forceinline__ unsigned long long sdesc(unsigned addr, unsigned lbo, unsigned sbo)
{
    return (unsigned long long)((addr & 0x3FFFFu) >> 4) | ((unsigned long long)((lbo >> 4) & 0x3FFFu) << 16) |
           ((unsigned long long)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: D FP32, A and B BF16, both K-major
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity)
{
    for (long long n = 0; n < SPIN_LIMIT; ++n) {
        unsigned ok;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(smem_u32(b)), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// byte offset of element (r, k) of a staged 64-wide K chunk
__device__ __forceinline__ int core_off(int r, int k) { return (((r >> 3) * 8 + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1); }

// Rows [r0, r0 + rows) x K columns [k0, k0 + 64) of X (element (r, k) at
// X[r s_r + k s_k]) into a stage in the core-matrix layout; rows at or beyond
// nrow and columns at or beyond K are zero.  rows is a multiple of 8, r0 and k0
// of 64.
__device__ __forceinline__ void stage_operand(const __nv_bfloat16* X, long long s_r, long long s_k, int r0, int rows,
                                              int nrow, int k0, int K, unsigned char* dst, int tid)
{
    const __nv_bfloat16 zero = __float2bfloat16(0.0f);
    const bool al = (reinterpret_cast<uintptr_t>(X) & 15u) == 0;
    if (s_k == 1 && al && (s_r & 7) == 0) {
        // K-major: 8 consecutive K per thread, one 16-byte load and store
        for (int idx = tid; idx < rows * (GK / 8); idx += GTHREADS) {
            const int r = idx / (GK / 8), kc = (idx % (GK / 8)) * 8;
            const int m = r0 + r, kk = k0 + kc;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (m < nrow) {
                if (kk + 8 <= K) {
                    v = __ldg(reinterpret_cast<const uint4*>(X + m * s_r + kk));
                } else {
                    unsigned w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        if (kk + j < K)
                            w[j >> 1] |= (unsigned)__bfloat16_as_ushort(X[m * s_r + kk + j]) << (16 * (j & 1));
                    v = make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            *reinterpret_cast<uint4*>(dst + core_off(r, kc)) = v;
        }
    } else if (s_r == 1 && al && (s_k & 7) == 0) {
        // transposed: 8 consecutive rows per thread, one 16-byte load, eight
        // 2-byte stores (the rows of a core matrix are 16 bytes apart)
        for (int idx = tid; idx < (rows / 8) * GK; idx += GTHREADS) {
            const int rc = (idx % (rows / 8)) * 8, k = idx / (rows / 8);
            const int m = r0 + rc, kk = k0 + k;
            unsigned w[4] = {0u, 0u, 0u, 0u};
            if (kk < K && m + 8 <= nrow) {
                const uint4 v = __ldg(reinterpret_cast<const uint4*>(X + m + kk * s_k));
                w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (kk < K && m + j < nrow)
                        w[j >> 1] |= (unsigned)__bfloat16_as_ushort(X[m + j + kk * s_k]) << (16 * (j & 1));
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                *reinterpret_cast<unsigned short*>(dst + core_off(rc + j, k)) = (unsigned short)(w[j >> 1] >> (16 * (j & 1)));
        }
    } else if (s_r == 1) {
        // transposed, unaligned: consecutive threads on consecutive rows
        for (int idx = tid; idx < rows * GK; idx += GTHREADS) {
            const int r = idx % rows, k = idx / rows;
            const int m = r0 + r, kk = k0 + k;
            *reinterpret_cast<__nv_bfloat16*>(dst + core_off(r, k)) = (m < nrow && kk < K) ? X[m + kk * s_k] : zero;
        }
    } else {
        for (int idx = tid; idx < rows * GK; idx += GTHREADS) {
            const int r = idx / GK, k = idx % GK;
            const int m = r0 + r, kk = k0 + k;
            *reinterpret_cast<__nv_bfloat16*>(dst + core_off(r, k)) =
                (m < nrow && kk < K) ? X[m * s_r + kk * s_k] : zero;
        }
    }
}

__global__ void __launch_bounds__(GTHREADS) gemm_kernel(const GemmArgs g)
{
    extern __shared__ __align__(128) unsigned char sm[];
    __shared__ unsigned long long bar;
    __shared__ unsigned s_tmem;
    // stage b: A at sm + b GEMM_STAGE, B SMEM_A after it
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    const int nrem = g.N - n0;
    const int nt = ((nrem < GN ? nrem : GN) + 15) & ~15;      // MMA N: multiple of 16
    const unsigned ncols = nt <= 32 ? 32u : (nt <= 64 ? 64u : (nt <= 128 ? 128u : 256u));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = s_tmem;
    const unsigned idesc = idesc_bf16(GM, nt);
    unsigned phase = 0;
    bool ok = true;
    const int nchunk = (g.K + GK - 1) / GK;
    stage_operand(g.A, g.a_sm, g.a_sk, m0, GM, g.M, 0, g.K, sm, tid);
    stage_operand(g.B, g.b_sn, g.b_sk, n0, nt, g.N, 0, g.K, sm + SMEM_A, tid);
    // generic-proxy writes of the stage before the tensor core reads them
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    for (int c = 0; c < nchunk; ++c) {
        unsigned char* sa = sm + (c & 1) * GEMM_STAGE;
        unsigned char* sb = sa + SMEM_A;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk) {
                const unsigned long long ad = sdesc(smem_u32(sa) + kk * 256u, 128u, 1024u);
                const unsigned long long bd = sdesc(smem_u32(sb) + kk * 256u, 128u, 1024u);
                const unsigned acc = (c > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar))
                         : "memory");
        }
        if (c + 1 < nchunk) {
            // the next chunk into the other stage while these products run
            unsigned char* na = sm + ((c + 1) & 1) * GEMM_STAGE;
            stage_operand(g.A, g.a_sm, g.a_sk, m0, GM, g.M, (c + 1) * GK, g.K, na, tid);
            stage_operand(g.B, g.b_sn, g.b_sk, n0, nt, g.N, (c + 1) * GK, g.K, na + SMEM_A, tid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        const bool got = mbar_wait(&bar, phase);
        phase ^= 1u;
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok) {
        // give the issued products a second bounded wait before freeing TMEM
        if (tid == 0) {
            atomicOr(&g_gemm_status, 1u);
            if (g.status) atomicOr(g.status, 1u);
        }
        (void)mbar_wait(&bar, phase ^ 1u);
    } else {
        const int m = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < nt; c0 += 16) {
            unsigned r[16];
            const unsigned ta = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < g.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n >= g.N) continue;
                    float v = __uint_as_float(r[j]);
                    if (g.bias) v += g.bias[n];
                    if (g.relu) v = fmaxf(v, 0.0f);
                    const long long o = m * g.c_sm + n * g.c_sn;
                    if (g.mask && !(__bfloat162float(g.mask[o]) > 0.0f)) v = 0.0f;
                    if (g.C32) g.C32[o] = v;
                    if (g.C16) g.C16[o] = __float2bfloat16(v);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

cudaError_t launch_gemm(const GemmArgs& g, cudaStream_t s)
{
    // the opt-in to 96 KiB of dynamic shared memory is per device: set it on
    // every launch (a cheap call) rather than once per process
    const cudaError_t e = cudaFuncSetAttribute(gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, GEMM_SMEM);
    if (e != cudaSuccess) return e;
    const dim3 grid((g.M + GM - 1) / GM, (g.N + GN - 1) / GN);
    gemm_kernel<<<grid, GTHREADS, GEMM_SMEM, s>>>(g);
    return cudaGetLastError();
}

}  // namespace lbsur

using namespace lbsur;

extern "C" lb_status lb_gemm_bf16(const uint16_t* A, int64_t a_sm, int64_t a_sk, const uint16_t* B, int64_t b_sn,
                                  int64_t b_sk, int32_t M, int32_t N, int32_t K, const float* bias, int32_t relu,
                                  float* C32, uint16_t* C16, int64_t c_sm, int64_t c_sn, void* stream)
{
    if (!A || !B || M < 1 || N < 1 || K < 1 || (!C32 && !C16)) return LB_EINVAL;
    GemmArgs g{};
    g.A = reinterpret_cast<const __nv_bfloat16*>(A);
    g.a_sm = a_sm; g.a_sk = a_sk;
    g.B = reinterpret_cast<const __nv_bfloat16*>(B);
    g.b_sn = b_sn; g.b_sk = b_sk;
    g.M = M; g.N = N; g.K = K;
    g.bias = bias; g.relu = relu;
    g.C32 = C32; g.C16 = reinterpret_cast<__nv_bfloat16*>(C16);
    g.c_sm = c_sm; g.c_sn = c_sn;
    return launch_gemm(g, static_cast<cudaStream_t>(stream)) == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_gemm_status(void)
{
    if (cudaDeviceSynchronize() != cudaSuccess) return LB_ECUDA;
    unsigned v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_gemm_status, sizeof(v)) != cudaSuccess) return LB_ECUDA;
    if (v && cudaMemcpyToSymbol(g_gemm_status, &z, sizeof(z)) != cudaSuccess) return LB_ECUDA;
    return v ? LB_ETIMEOUT : LB_OK;
}

// ---------------------------------------------------------------------------
// The network: parameters, activations and the kernels around the products.
namespace lbsur {

constexpr int NIN = LB_MLP_IN, NINP = LB_MLP_IN_PAD, NH = LB_MLP_HID, NOUT = LB_MLP_OUT, NOUTP = LB_MLP_OUT_PAD;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NINP, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUTP * NH, NPARAM = OFF_B3 + NOUTP;
static_assert(NPARAM == LB_MLP_NPARAM, "parameter layout");

// lower-triangle index t of (i, j), j <= i: t = i (i + 1) / 2 + j
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

__global__ void features_kernel(const float* x, int n, __nv_bfloat16* X)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * NINP) return;
    const int s = idx / NINP, k = idx % NINP;
    X[idx] = __float2bfloat16(k < NIN ? x[s * NIN + k] : 0.0f);
}

__global__ void to_bf16_kernel(const float* p, __nv_bfloat16* q, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) q[i] = __float2bfloat16(p[i]);
}

__device__ __forceinline__ float softplus(float y) { return y > 20.0f ? y : log1pf(expf(y)); }
__device__ __forceinline__ float sigmoid(float y) { return 1.0f / (1.0f + expf(-y)); }

// Output head, one thread per sample: L from the 21 outputs (diagonal through
// softplus), R^ = L L^T; with targets, the loss (1/(36 n)) sum (R^ - Rt)^2 and
// its gradient with respect to the outputs: dR = 2 (R^ - Rt) / (36 n),
// dL = 2 dR L (dR symmetric), dy = dL (off the diagonal), dL_ii sigmoid(y_ii).
__global__ void head_kernel(const float* Y, int n, float* y_out, float* R_out, const float* Rt, float* loss,
                            float* dY32, __nv_bfloat16* dY16)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    float part = 0.0f;
    if (s < n) {
        float y[NOUT], L[6][6], R[6][6];
#pragma unroll
        for (int t = 0; t < NOUT; ++t) y[t] = Y[s * NOUTP + t];
        if (y_out) {
            for (int t = 0; t < NOUT; ++t) y_out[s * NOUT + t] = y[t];
        }
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < 6; ++j) L[i][j] = j < i ? y[tri(i, j)] : (j == i ? softplus(y[tri(i, i)]) : 0.0f);
#pragma unroll
        for (int i = 0; i < 6; ++i)
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                float a = 0.0f;
#pragma unroll
                for (int k = 0; k < 6; ++k) a += L[i][k] * L[j][k];
                R[i][j] = a;
            }
        if (R_out) {
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) R_out[s * 36 + i * 6 + j] = R[i][j];
        }
        if (Rt) {
            const float c = 2.0f / (36.0f * (float)n);
            float dR[6][6];
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    const float d = R[i][j] - Rt[s * 36 + i * 6 + j];
                    part += d * d;
                    dR[i][j] = c * d;
                }
            float dy[NOUTP];
#pragma unroll
            for (int t = 0; t < NOUTP; ++t) dy[t] = 0.0f;
#pragma unroll
            for (int i = 0; i < 6; ++i)
#pragma unroll
                for (int j = 0; j <= i; ++j) {
                    float a = 0.0f;
#pragma unroll
                    for (int k = 0; k < 6; ++k) a += dR[i][k] * L[k][j];
                    a *= 2.0f;
                    dy[tri(i, j)] = (j == i) ? a * sigmoid(y[tri(i, i)]) : a;
                }
#pragma unroll
            for (int t = 0; t < NOUTP; ++t) {
                dY32[s * NOUTP + t] = dy[t];
                dY16[s * NOUTP + t] = __float2bfloat16(dy[t]);
            }
        }
    }
    if (Rt) {
        // block sum of the squared errors, one atomic per block
        __shared__ float red[32];
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
        __syncthreads();
        if (threadIdx.x < 32) {
            float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) atomicAdd(loss, v / (36.0f * (float)n));
        }
    }
}

// column sums of an FP32 [n][w] matrix (bias gradients), one thread per column
__global__ void colsum_kernel(const float* D, int n, int w, float* out)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= w) return;
    float a = 0.0f;
    for (int s = 0; s < n; ++s) a += D[(long long)s * w + c];
    out[c] = a;
}

__global__ void adam_kernel(float* p, const float* g, float* m1, float* m2, int n, float lr, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = 0.9f * m1[i] + 0.1f * gi;
    const float b = 0.999f * m2[i] + 0.001f * gi * gi;
    m1[i] = a;
    m2[i] = b;
    p[i] -= lr * (a * c1) / (sqrtf(b * c2) + 1e-8f);
}

// Cholesky solve of A u = f for one symmetric positive definite 6x6 A (FP64,
// A overwritten)
__device__ void chol_solve6(double (&A)[6][6], const double* f, double* u)
{
    double y[6];
    for (int j = 0; j < 6; ++j) {                      // A = C C^T, C lower, in place
        double d = A[j][j];
        for (int k = 0; k < j; ++k) d -= A[j][k] * A[j][k];
        d = d > 0.0 ? sqrt(d) : 0.0;
        A[j][j] = d;
        for (int i = j + 1; i < 6; ++i) {
            double a = A[i][j];
            for (int k = 0; k < j; ++k) a -= A[i][k] * A[j][k];
            A[i][j] = d > 0.0 ? a / d : 0.0;
        }
    }
    for (int i = 0; i < 6; ++i) {
        double a = f[i];
        for (int k = 0; k < i; ++k) a -= A[i][k] * y[k];
        y[i] = A[i][i] > 0.0 ? a / A[i][i] : 0.0;
    }
    for (int i = 5; i >= 0; --i) {
        double a = y[i];
        for (int k = i + 1; k < 6; ++k) a -= A[k][i] * u[k];
        u[i] = A[i][i] > 0.0 ? a / A[i][i] : 0.0;
    }
}

// Cholesky solve of R u = f per sample, FP64 (R read as FP32, symmetrised)
__global__ void spd_solve_kernel(const float* R, const double* f, double* u, int n)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double A[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i][j] = 0.5 * ((double)R[s * 36 + i * 6 + j] + (double)R[s * 36 + j * 6 + i]);
    chol_solve6(A, f + s * 6, u + s * 6);
}

// inverse of a 6x6 matrix M (Gauss-Jordan with partial pivoting, FP64),
// symmetrised, into out
__device__ void invert6_sym(const double* M, double* out)
{
    double A[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j) A[i][j] = j < 6 ? M[i * 6 + j] : (j - 6 == i ? 1.0 : 0.0);
    for (int c = 0; c < 6; ++c) {
        int piv = c;
        for (int r = c + 1; r < 6; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (piv != c)
            for (int j = 0; j < 12; ++j) { const double t = A[c][j]; A[c][j] = A[piv][j]; A[piv][j] = t; }
        const double d = A[c][c];
        const double id = d != 0.0 ? 1.0 / d : 0.0;
        for (int j = 0; j < 12; ++j) A[c][j] *= id;
        for (int r = 0; r < 6; ++r) {
            if (r == c) continue;
            const double fct = A[r][c];
            for (int j = 0; j < 12; ++j) A[r][j] -= fct * A[c][j];
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) out[i * 6 + j] = 0.5 * (A[i][j + 6] + A[j][i + 6]);
}

__global__ void spd_invert_kernel(double* M, int n)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double t[36];
    invert6_sym(M + s * 36, t);
    for (int k = 0; k < 36; ++k) M[s * 36 + k] = t[k];
}

// ---- features and scaling of the resistance tensor.  geom per sample:
// (a, b, nu, L, e_x, e_y, e_z, rho0): semi-axes a (along the unit long axis e)
// and b, kinematic viscosity, box edge (or the edge of the volume per
// particle), fluid density.  D = diag(s_t I3, s_r I3) with s_t^2 = 6 pi mu b and
// s_r^2 = 8 pi mu b^3 (mu = rho0 nu): the radius-b sphere's Stokes resistances,
// so that R^ = D^-1 R D^-1 is the identity for that sphere in free space.
__device__ __forceinline__ void scales(const double* g, double& st, double& sr)
{
    const double mu = g[7] * g[2], b = g[1];
    st = sqrt(6.0 * M_PI * mu * b);
    sr = sqrt(8.0 * M_PI * mu * b * b * b);
}

__global__ void features_geom_kernel(const double* geom, int n, float* x)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const double* g = geom + s * 8;
    const double sg = g[6] < 0.0 ? -1.0 : 1.0;       // head-tail symmetry: e and -e are the same spheroid
    x[s * 8 + 0] = (float)(g[0] / g[1] - 2.0);
    x[s * 8 + 1] = (float)(g[1] - 3.0);
    x[s * 8 + 2] = (float)((g[2] - 1.0 / 6.0) * 10.0);
    x[s * 8 + 3] = (float)(g[1] / g[3] * 10.0 - 1.0);
    x[s * 8 + 4] = (float)(sg * g[4]);
    x[s * 8 + 5] = (float)(sg * g[5]);
    x[s * 8 + 6] = (float)(sg * g[6]);
    x[s * 8 + 7] = 1.0f;
}

// measured mobility M (6x6, FP64) -> R^ = (D M D)^-1 (FP32)
__global__ void targets_kernel(const double* M, const double* geom, int n, float* Rhat)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double st, sr;
    scales(geom + s * 8, st, sr);
    double A[36], t[36];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i * 6 + j] = (i < 3 ? st : sr) * M[s * 36 + i * 6 + j] * (j < 3 ? st : sr);
    invert6_sym(A, t);
    for (int k = 0; k < 36; ++k) Rhat[s * 36 + k] = (float)t[k];
}

// (U, Omega) = R^-1 (F, T) = D^-1 R^^-1 D^-1 (F, T)
__global__ void warm_velocities_kernel(const float* Rhat, const double* geom, const double* FT, int n, double* UW)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    double st, sr;
    scales(geom + s * 8, st, sr);
    double A[6][6], f[6], u[6];
    for (int i = 0; i < 6; ++i) {
        f[i] = FT[s * 6 + i] / (i < 3 ? st : sr);
        for (int j = 0; j < 6; ++j)
            A[i][j] = 0.5 * ((double)Rhat[s * 36 + i * 6 + j] + (double)Rhat[s * 36 + j * 6 + i]);
    }
    chol_solve6(A, f, u);
    for (int i = 0; i < 6; ++i) UW[s * 6 + i] = u[i] / (i < 3 ? st : sr);
}

}  // namespace lbsur

struct lb_mlp {
    int device = 0;
    int max_batch = 0;
    long long step = 0;
    float* p = nullptr;                 // FP32 master parameters
    float* g = nullptr;                 // gradients
    float* m1 = nullptr;                // Adam moments
    float* m2 = nullptr;
    float* loss = nullptr;              // scratch loss for train_step without output
    __nv_bfloat16* w16 = nullptr;       // BF16 copy of the whole parameter block (W1, W2, W3 used)
    __nv_bfloat16* X = nullptr;         // [B][16]
    __nv_bfloat16* H1 = nullptr;        // [B][256]
    __nv_bfloat16* H2 = nullptr;
    float* Y = nullptr;                 // [B][32]
    float* dY32 = nullptr;
    __nv_bfloat16* dY16 = nullptr;
    float* dH32 = nullptr;              // [B][256], reused for both hidden layers
    __nv_bfloat16* dH2 = nullptr;
    __nv_bfloat16* dH1 = nullptr;
    std::vector<void*> allocs;
};

namespace {

template <class T>
bool mlp_alloc(lb_mlp* m, T** p, size_t count)
{
    void* q = nullptr;
    if (cudaMalloc(&q, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    m->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return true;
}

void mlp_free(lb_mlp* m)
{
    for (void* q : m->allocs) cudaFree(q);
    m->allocs.clear();
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

GemmArgs gemm(const __nv_bfloat16* A, long long a_sm, long long a_sk, const __nv_bfloat16* B, long long b_sn,
              long long b_sk, int M, int N, int K)
{
    GemmArgs g{};
    g.A = A; g.a_sm = a_sm; g.a_sk = a_sk;
    g.B = B; g.b_sn = b_sn; g.b_sk = b_sk;
    g.M = M; g.N = N; g.K = K;
    return g;
}

// forward pass of n samples into m->H1, m->H2, m->Y
cudaError_t forward(lb_mlp* m, const float* x, int n, cudaStream_t s)
{
    cudaError_t e;
    features_kernel<<<blocks((long long)n * NINP, 256), 256, 0, s>>>(x, n, m->X);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    GemmArgs g = gemm(m->X, NINP, 1, m->w16 + OFF_W1, NINP, 1, n, NH, NINP);
    g.bias = m->p + OFF_B1; g.relu = 1; g.C16 = m->H1; g.c_sm = NH; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    g = gemm(m->H1, NH, 1, m->w16 + OFF_W2, NH, 1, n, NH, NH);
    g.bias = m->p + OFF_B2; g.relu = 1; g.C16 = m->H2; g.c_sm = NH; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    g = gemm(m->H2, NH, 1, m->w16 + OFF_W3, NH, 1, n, NOUTP, NH);
    g.bias = m->p + OFF_B3; g.C32 = m->Y; g.c_sm = NOUTP; g.c_sn = 1;
    return launch_gemm(g, s);
}

// loss and gradients into m->g (after forward); loss accumulated into `loss`
cudaError_t backward(lb_mlp* m, const float* Rt, int n, float* loss, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(float), s)) != cudaSuccess) return e;
    head_kernel<<<blocks(n, 128), 128, 0, s>>>(m->Y, n, nullptr, nullptr, Rt, loss, m->dY32, m->dY16);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // layer 3: dW3 = dY^T H2, db3 = sum dY
    GemmArgs g = gemm(m->dY16, 1, NOUTP, m->H2, 1, NH, NOUTP, NH, n);
    g.C32 = m->g + OFF_W3; g.c_sm = NH; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    colsum_kernel<<<1, NOUTP, 0, s>>>(m->dY32, n, NOUTP, m->g + OFF_B3);
    // dH2 = (dY W3) * [H2 > 0]
    g = gemm(m->dY16, NOUTP, 1, m->w16 + OFF_W3, 1, NH, n, NH, NOUTP);
    g.mask = m->H2; g.C32 = m->dH32; g.C16 = m->dH2; g.c_sm = NH; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    colsum_kernel<<<1, NH, 0, s>>>(m->dH32, n, NH, m->g + OFF_B2);
    // layer 2: dW2 = dH2^T H1
    g = gemm(m->dH2, 1, NH, m->H1, 1, NH, NH, NH, n);
    g.C32 = m->g + OFF_W2; g.c_sm = NH; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    // dH1 = (dH2 W2) * [H1 > 0]
    g = gemm(m->dH2, NH, 1, m->w16 + OFF_W2, 1, NH, n, NH, NH);
    g.mask = m->H1; g.C32 = m->dH32; g.C16 = m->dH1; g.c_sm = NH; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    colsum_kernel<<<1, NH, 0, s>>>(m->dH32, n, NH, m->g + OFF_B1);
    // layer 1: dW1 = dH1^T X
    g = gemm(m->dH1, 1, NH, m->X, 1, NINP, NH, NINP, n);
    g.C32 = m->g + OFF_W1; g.c_sm = NINP; g.c_sn = 1;
    if ((e = launch_gemm(g, s)) != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t refresh_bf16(lb_mlp* m, cudaStream_t s)
{
    to_bf16_kernel<<<blocks(NPARAM, 256), 256, 0, s>>>(m->p, m->w16, NPARAM);
    return cudaGetLastError();
}

}  // namespace

extern "C" lb_status lb_mlp_create(int32_t device, int32_t max_batch, lb_mlp** out)
{
    if (!out || max_batch < 1 || max_batch > LB_MLP_MAX_BATCH) return LB_EINVAL;
    *out = nullptr;
    if (cudaSetDevice(device) != cudaSuccess) return LB_ECUDA;
    lb_mlp* m = new (std::nothrow) lb_mlp;
    if (!m) return LB_ENOMEM;
    m->device = device;
    m->max_batch = max_batch;
    const size_t B = (size_t)max_batch;
    bool ok = mlp_alloc(m, &m->p, NPARAM) && mlp_alloc(m, &m->g, NPARAM) && mlp_alloc(m, &m->m1, NPARAM) &&
              mlp_alloc(m, &m->m2, NPARAM) && mlp_alloc(m, &m->loss, 1) && mlp_alloc(m, &m->w16, NPARAM) &&
              mlp_alloc(m, &m->X, B * NINP) && mlp_alloc(m, &m->H1, B * NH) && mlp_alloc(m, &m->H2, B * NH) &&
              mlp_alloc(m, &m->Y, B * NOUTP) && mlp_alloc(m, &m->dY32, B * NOUTP) &&
              mlp_alloc(m, &m->dY16, B * NOUTP) && mlp_alloc(m, &m->dH32, B * NH) && mlp_alloc(m, &m->dH2, B * NH) &&
              mlp_alloc(m, &m->dH1, B * NH);
    if (ok) {
        for (void* q : {(void*)m->p, (void*)m->g, (void*)m->m1, (void*)m->m2})
            ok = ok && cudaMemset(q, 0, NPARAM * sizeof(float)) == cudaSuccess;
        ok = ok && cudaMemset(m->w16, 0, NPARAM * sizeof(__nv_bfloat16)) == cudaSuccess;
        ok = ok && cudaDeviceSynchronize() == cudaSuccess;
    }
    if (!ok) {
        mlp_free(m);
        delete m;
        return LB_ENOMEM;
    }
    *out = m;
    return LB_OK;
}

extern "C" lb_status lb_mlp_destroy(lb_mlp* m)
{
    if (!m) return LB_EINVAL;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    mlp_free(m);
    delete m;
    return LB_OK;
}

extern "C" lb_status lb_mlp_set_params(lb_mlp* m, const float* host)
{
    if (!m || !host) return LB_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return LB_ECUDA;
    std::vector<float> h(host, host + NPARAM);
    // padding stays zero: W1 columns 8..15, W3 rows and b3 entries 21..31
    for (int r = 0; r < NH; ++r)
        for (int c = NIN; c < NINP; ++c) h[OFF_W1 + r * NINP + c] = 0.0f;
    for (int r = NOUT; r < NOUTP; ++r) {
        for (int c = 0; c < NH; ++c) h[OFF_W3 + r * NH + c] = 0.0f;
        h[OFF_B3 + r] = 0.0f;
    }
    if (cudaMemcpy(m->p, h.data(), NPARAM * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(m->m1, 0, NPARAM * sizeof(float)) != cudaSuccess ||
        cudaMemset(m->m2, 0, NPARAM * sizeof(float)) != cudaSuccess || refresh_bf16(m, nullptr) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess)
        return LB_ECUDA;
    m->step = 0;
    return LB_OK;
}

extern "C" lb_status lb_mlp_get_params(lb_mlp* m, float* host)
{
    if (!m || !host) return LB_EINVAL;
    if (cudaSetDevice(m->device) != cudaSuccess) return LB_ECUDA;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(host, m->p, NPARAM * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return LB_ECUDA;
    return LB_OK;
}

extern "C" lb_status lb_mlp_forward(lb_mlp* m, const float* x_dev, int32_t n, float* y_dev, float* R_dev, void* stream)
{
    if (!m || !x_dev || n < 1 || n > m->max_batch) return LB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(m->device) != cudaSuccess || forward(m, x_dev, n, s) != cudaSuccess) return LB_ECUDA;
    head_kernel<<<blocks(n, 128), 128, 0, s>>>(m->Y, n, y_dev, R_dev, nullptr, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_mlp_loss_grad(lb_mlp* m, const float* x_dev, const float* Rt_dev, int32_t n, float* loss_dev,
                                      float* grad_dev, void* stream)
{
    if (!m || !x_dev || !Rt_dev || !loss_dev || n < 1 || n > m->max_batch) return LB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(m->device) != cudaSuccess || forward(m, x_dev, n, s) != cudaSuccess ||
        backward(m, Rt_dev, n, loss_dev, s) != cudaSuccess)
        return LB_ECUDA;
    if (grad_dev && cudaMemcpyAsync(grad_dev, m->g, NPARAM * sizeof(float), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return LB_ECUDA;
    return LB_OK;
}

extern "C" lb_status lb_mlp_train_step(lb_mlp* m, const float* x_dev, const float* Rt_dev, int32_t n, float lr,
                                       float* loss_dev, void* stream)
{
    if (!m || !x_dev || !Rt_dev || n < 1 || n > m->max_batch || !(lr > 0.0f)) return LB_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaSetDevice(m->device) != cudaSuccess || forward(m, x_dev, n, s) != cudaSuccess ||
        backward(m, Rt_dev, n, loss_dev ? loss_dev : m->loss, s) != cudaSuccess)
        return LB_ECUDA;
    m->step += 1;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)m->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)m->step)));
    adam_kernel<<<blocks(NPARAM, 256), 256, 0, s>>>(m->p, m->g, m->m1, m->m2, NPARAM, lr, c1, c2);
    if (cudaGetLastError() != cudaSuccess || refresh_bf16(m, s) != cudaSuccess) return LB_ECUDA;
    return LB_OK;
}

extern "C" lb_status lb_spd_solve6(const float* R_dev, const double* f_dev, double* u_dev, int32_t n, void* stream)
{
    if (!R_dev || !f_dev || !u_dev || n < 1) return LB_EINVAL;
    spd_solve_kernel<<<blocks(n, 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(R_dev, f_dev, u_dev, n);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_spd_invert6(double* M_dev, int32_t n, void* stream)
{
    if (!M_dev || n < 1) return LB_EINVAL;
    spd_invert_kernel<<<blocks(n, 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(M_dev, n);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_mlp_features(const double* geom_dev, int32_t n, float* x_dev, void* stream)
{
    if (!geom_dev || !x_dev || n < 1) return LB_EINVAL;
    features_geom_kernel<<<blocks(n, 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(geom_dev, n, x_dev);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_resistance_targets(const double* M_dev, const double* geom_dev, int32_t n, float* Rhat_dev,
                                           void* stream)
{
    if (!M_dev || !geom_dev || !Rhat_dev || n < 1) return LB_EINVAL;
    targets_kernel<<<blocks(n, 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(M_dev, geom_dev, n, Rhat_dev);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

extern "C" lb_status lb_warm_velocities(const float* Rhat_dev, const double* geom_dev, const double* FT_dev, int32_t n,
                                        double* UW_dev, void* stream)
{
    if (!Rhat_dev || !geom_dev || !FT_dev || !UW_dev || n < 1) return LB_EINVAL;
    warm_velocities_kernel<<<blocks(n, 64), 64, 0, static_cast<cudaStream_t>(stream)>>>(Rhat_dev, geom_dev, FT_dev, n,
                                                                                         UW_dev);
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}
