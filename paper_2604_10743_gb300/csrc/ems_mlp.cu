// ems_mlp.cu -- the surrogate's multilayer perceptron on the tensor cores.
//
// Training: every dense layer is one tcgen05 GEMM (BF16 operands, FP32
// accumulation in tensor memory) with the bias / ReLU / ReLU'-mask epilogue
// fused; the backward pass is two GEMMs per layer (dW = dZ^T H and
// dH = dZ W, both K-major thanks to transposed copies the forward epilogue
// writes) plus a column sum for db; Adam runs on FP32 master weights and
// refreshes the BF16 copies.
//
// Inference: one persistent kernel runs all layers for 256 rows per CTA.  The
// activations never leave shared memory; the weights stream from L2 in 16 KB
// chunks that are stored in global memory already in the tensor core's
// 128-byte swizzled layout, so each chunk is one cp.async.bulk copy into a
// six-stage ring.  Thread 0 issues the MMAs (two 128-row accumulators, 512
// TMEM columns) and all eight warps run the epilogues.
//
// Operand layout in shared memory (K-major, 128-byte swizzle): a tile of R
// rows x 64 BF16 (one "K chunk") stores row r's 16-byte unit u at byte
// r * 128 + ((u ^ (r & 7)) << 4); eight rows form a 1024-byte atom.  All
// operand buffers are 1024-byte aligned.  Every mbarrier wait is bounded and
// reports a timeout through the status word instead of hanging.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "ems_internal.cuh"
#include "../../include/ems_surrogate.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int NF = EMS_MLP_FEATURES, NO = EMS_MLP_OUTPUTS, WID = EMS_MLP_WIDTH;
constexpr int MAXL = 9;                       // layers: up to 8 hidden + head
constexpr long long kWaitCycles = 1LL << 32;  // SM clocks an mbarrier wait may take (~2 s)
constexpr int kStTimeout = 1;                 // status word: a wait gave up

// ---------------------------------------------------------------------------
// tcgen05 / mbarrier / bulk-copy primitives (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// matrix descriptor: K-major, 128-byte swizzle, 1024-byte stride between
// 8-row atoms, descriptor version 1
__device__ __forceinline__ uint64_t sdesc(uint32_t a) {
    return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor of kind::f16: BF16 A and B, FP32 D, both K-major,
// M = 128, N = n (multiple of 16, <= 256)
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count));
}

// Wait for the phase with the given parity.  Each try suspends the thread
// for at most 1 us (the hardware wakes it earlier when the phase completes);
// after about two seconds of SM clock the wait gives up and flags a timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int32_t *status) {
    const uint32_t a = saddr(bar);
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(1000u)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) break;
    }
    atomicOr(&status[kStTimeout], 1);
    return false;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// ---------------------------------------------------------------------------
// Training GEMM: D[M x N] = scale * A[M x K] B[N x K]^T, fused epilogue
// ---------------------------------------------------------------------------
constexpr int GBM = 128, GBK = 64;
constexpr int G_A_BYTES = GBM * GBK * 2;            // 16 KB
constexpr int G_B_BYTES = 256 * GBK * 2;            // 32 KB
constexpr int G_STAGE = G_A_BYTES + G_B_BYTES;
constexpr int G_SMEM = 2 * G_STAGE + 1024;

struct GemmArgs {
    const bf16 *A, *B;
    int M, N, K;
    const float *bias;      // [N] or null
    const bf16 *mask;       // [M x N] or null: zero where mask <= 0 (ReLU')
    float *out_f32;         // [M x N] or null
    bf16 *out_bf16;         // [M x N] or null
    bf16 *out_t;            // [N x ldt] or null: transposed BF16 copy
    int ldt;
    int relu;
    float scale;
    int32_t *status;
};

// One CTA per 128-row tile; two stages of 64-wide K chunks of A and B staged
// through registers into the swizzled layout, MMAs of chunk k overlapping the
// loads of chunk k + 1.
__global__ void __launch_bounds__(128, 1) k_gemm_tc(GemmArgs g) {
    extern __shared__ uint8_t smraw[];
    __shared__ uint64_t mbar[2];
    __shared__ uint32_t tmem_slot;
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * GBM;
    const int nk = g.K / GBK;
    const uint32_t idesc = idesc_bf16(g.N);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;
    bool ok = true;
    int issued = 0;

    for (int kc = 0; kc < nk; ++kc) {
        const int buf = kc & 1;
        uint8_t *sA = sm + buf * G_STAGE, *sB = sA + G_A_BYTES;
        if (kc >= 2) ok = mbar_wait(&mbar[buf], ((kc - 2) >> 1) & 1, g.status);
        if (!__syncthreads_and(ok)) { ok = false; break; }
        const int kbase = kc * GBK;
        for (int q = tid; q < GBM * 8; q += 128) {
            const int r = q >> 3, u = q & 7, gr = m0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < g.M) v = *(const uint4 *)(g.A + (int64_t)gr * g.K + kbase + u * 8);
            *(uint4 *)(sA + r * 128 + ((u ^ (r & 7)) << 4)) = v;
        }
        for (int q = tid; q < g.N * 8; q += 128) {
            const int r = q >> 3, u = q & 7;
            const uint4 v = *(const uint4 *)(g.B + (int64_t)r * g.K + kbase + u * 8);
            *(uint4 *)(sB + r * 128 + ((u ^ (r & 7)) << 4)) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
            for (int kk = 0; kk < GBK / 16; ++kk)
                mma_bf16(tmem, sdesc(saddr(sA + kk * 32)), sdesc(saddr(sB + kk * 32)), idesc, (kc | kk) ? 1u : 0u);
            mma_commit(&mbar[buf]);
        }
        issued = kc + 1;
    }
    // the last commit covers every MMA issued before it
    if (issued > 0) {
        const bool fin = mbar_wait(&mbar[(issued - 1) & 1], ((issued - 1) >> 1) & 1, g.status);
        ok = ok && fin;
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (__syncthreads_and(ok)) {
        const int lr = warp * 32 + lane, row = m0 + lr;
        for (int c0 = 0; c0 < g.N; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            if (row >= g.M) continue;
            const int nv = min(32, g.N - c0);
            const int64_t o = (int64_t)row * g.N + c0;
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                float x = __uint_as_float(r[j]) * g.scale;
                if (g.bias && j < nv) x += g.bias[c0 + j];
                if (g.relu) x = fmaxf(x, 0.0f);
                v[j] = x;
            }
            if (g.mask) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (q * 8 >= nv) break;
                    const uint4 mv = *(const uint4 *)(g.mask + o + q * 8);
                    const bf16 *mb = reinterpret_cast<const bf16 *>(&mv);
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (!(__bfloat162float(mb[e]) > 0.0f)) v[q * 8 + e] = 0.0f;
                }
            }
            if (g.out_f32) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q * 4 < nv)
                        *(float4 *)(g.out_f32 + o + q * 4) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
            if (g.out_bf16) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (q * 8 < nv)
                        *(uint4 *)(g.out_bf16 + o + q * 8) =
                            make_uint4(pack2(v[8 * q], v[8 * q + 1]), pack2(v[8 * q + 2], v[8 * q + 3]),
                                       pack2(v[8 * q + 4], v[8 * q + 5]), pack2(v[8 * q + 6], v[8 * q + 7]));
            }
            if (g.out_t) {
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < nv) g.out_t[(int64_t)(c0 + j) * g.ldt + row] = __float2bfloat16(v[j]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

bool gemm_shape_ok(int M, int N, int K) { return M >= 1 && N >= 16 && N <= 256 && N % 16 == 0 && K >= 64 && K % 64 == 0; }

cudaError_t launch_gemm(cudaStream_t st, const GemmArgs &g) {
    cudaError_t e = cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, G_SMEM);
    if (e != cudaSuccess) return e;
    k_gemm_tc<<<(g.M + GBM - 1) / GBM, 128, G_SMEM, st>>>(g);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused inference: all layers, 256 rows per CTA, weights streamed by TMA bulk
// copies from a pre-swizzled image.  Warp roles:
//   warps 0-7  epilogue: warp w owns TMEM lanes 32 (w % 4).. of tile w / 4
//              (layer-0 input, bias + ReLU -> BF16 operand, head output)
//   warp 8     producer: keeps the F_NS-stage weight ring full
//   warp 9     MMA issuer: tcgen05.mma of both tiles per weight chunk
// Hand-offs: full/empty (ring), done (MMAs of a layer finished -> epilogue),
// aready (next layer's A operand written and TMEM drained -> MMA).
// ---------------------------------------------------------------------------
constexpr int F_ROWS = 256;                   // rows per CTA (two 128-row accumulators)
constexpr int F_NS = 6;                       // weight-chunk ring stages
constexpr int F_CHUNK = 128 * 128;            // bytes of one 128-row x 64-K chunk
constexpr int F_A_TILE = 128 * 256 * 2;       // one tile's activations: 4 K chunks of 16 KB
constexpr int F_SMEM = 2 * F_A_TILE + F_NS * F_CHUNK + 1024;
constexpr int F_MAXCH = 64;
constexpr int F_THREADS = 320;

struct FusedArgs {
    const float *x;          // [rows][24]
    float *y;                // [rows][2]
    int64_t rows;
    int n_layers, n_chunks;
    const uint8_t *img;      // weight image
    const float *master;     // FP32 parameters (biases read from here)
    int boff[MAXL];          // bias offset of each layer in master (multiple of 4)
    int nout[MAXL];          // output width of each layer (2 for the head)
    int chunk_off[F_MAXCH];  // byte offset of each chunk in the image
    int chunk_info[F_MAXCH]; // layer << 16 | half << 8 | kc
    const float *norm;       // x mean[24], x std[24], t mean[2], t std[2]
    int32_t *status;
};

__device__ __forceinline__ int chunk_rows(const FusedArgs &a, int info) {
    const int l = info >> 16;
    return a.nout[l] >= 128 ? 128 : ((a.nout[l] + 15) & ~15);
}

__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}

__global__ void __launch_bounds__(F_THREADS, 1) k_mlp_fused(const __grid_constant__ FusedArgs a) {
    extern __shared__ uint8_t smraw[];
    __shared__ uint64_t full[F_NS], empty[F_NS], done, aready, fin;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int s_abort;
    __shared__ float s_norm[2 * NF + 2 * NO];
    uint8_t *sm = (uint8_t *)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
    uint8_t *sAct = sm;                          // [2 tiles][4 K chunks][128 rows x 128 B]
    uint8_t *sRing = sm + 2 * F_A_TILE;          // [F_NS][16 KB]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t n_pairs = (a.rows + F_ROWS - 1) / F_ROWS;
    const int64_t my_pairs = blockIdx.x < n_pairs ? (n_pairs - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t total = my_pairs * a.n_chunks;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_slot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int s = 0; s < F_NS; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        mbar_init(&aready, 256);
        mbar_init(&fin, 1);
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_abort = 0;
    }
    if (tid < 2 * NF + 2 * NO) s_norm[tid] = a.norm[tid];
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_slot;

    if (warp == 8) {
        // ---- producer: one bulk copy per weight chunk, F_NS in flight ----
        if (lane == 0) {
            int64_t g = 0;
            for (; g < total && !s_abort; ++g) {
                const int b = (int)(g % F_NS);
                if (g >= F_NS && !mbar_wait(&empty[b], (uint32_t)((g / F_NS - 1) & 1), a.status)) {
                    s_abort = 1;
                    break;
                }
                const int c = (int)(g % a.n_chunks);
                const uint32_t bytes = (uint32_t)chunk_rows(a, a.chunk_info[c]) * 128u;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(&full[b])),
                             "r"(bytes)
                             : "memory");
                asm volatile(
                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                        saddr(sRing + b * F_CHUNK)),
                    "l"(a.img + a.chunk_off[c]), "r"(bytes), "r"(saddr(&full[b]))
                    : "memory");
            }
            // every copy issued must land before the CTA may exit
            for (int64_t q = (g > F_NS ? g - F_NS : 0); q < g; ++q)
                mbar_wait(&full[q % F_NS], (uint32_t)((q / F_NS) & 1), a.status);
        }
        __syncwarp();
    } else if (warp == 9) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int64_t gq = 0;
            uint32_t lphase = 0;
            bool issued_any = false;
            for (int64_t pi = 0; pi < my_pairs && !s_abort; ++pi) {
                int c = 0;
                for (int l = 0; l < a.n_layers && !s_abort; ++l) {
                    if (!mbar_wait(&aready, lphase, a.status)) { s_abort = 1; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    while (c < a.n_chunks && (a.chunk_info[c] >> 16) == l) {
                        const int info = a.chunk_info[c];
                        const int h = (info >> 8) & 0xFF, kc = info & 0xFF;
                        const int b = (int)(gq % F_NS);
                        if (!mbar_wait(&full[b], (uint32_t)((gq / F_NS) & 1), a.status)) { s_abort = 1; break; }
                        const uint32_t id = idesc_bf16(chunk_rows(a, info));
                        const uint8_t *wb = sRing + b * F_CHUNK;
#pragma unroll
                        for (int t2 = 0; t2 < 2; ++t2) {
                            const uint8_t *ab = sAct + t2 * F_A_TILE + kc * F_CHUNK;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                mma_bf16(tmem + (uint32_t)(t2 * 256 + h * 128), sdesc(saddr(ab + kk * 32)),
                                         sdesc(saddr(wb + kk * 32)), id, (kc | kk) ? 1u : 0u);
                        }
                        issued_any = true;
                        mma_commit(&empty[b]);
                        ++gq;
                        ++c;
                    }
                    if (s_abort) break;
                    mma_commit(&done);
                    lphase ^= 1u;
                }
            }
            if (issued_any) {
                // the tensor core must be idle before TMEM is freed
                mma_commit(&fin);
                mbar_wait(&fin, 0, a.status);
            }
        }
        __syncwarp();
    } else {
        // ---- epilogue warps ----
        const int tile = warp >> 2, lq = warp & 3, lr = lq * 32 + lane;
        uint8_t *myA = sAct + tile * F_A_TILE;
        const uint32_t trow = tmem + ((uint32_t)(lq * 32) << 16) + (uint32_t)(tile * 256);
        uint32_t dphase = 0;
        for (int64_t pi = 0; pi < my_pairs && !s_abort; ++pi) {
            const int64_t row = (blockIdx.x + pi * gridDim.x) * F_ROWS + tile * 128 + lr;
            // layer-0 input: standardised features as BF16 in K chunk 0
            {
                float f[NF];
                if (row < a.rows) {
                    const float4 *xp = reinterpret_cast<const float4 *>(a.x + row * NF);
#pragma unroll
                    for (int q = 0; q < NF / 4; ++q) {
                        const float4 v = __ldg(xp + q);
                        f[4 * q] = v.x; f[4 * q + 1] = v.y; f[4 * q + 2] = v.z; f[4 * q + 3] = v.w;
                    }
#pragma unroll
                    for (int k = 0; k < NF; ++k) f[k] = (f[k] - s_norm[k]) / s_norm[NF + k];
                } else {
#pragma unroll
                    for (int k = 0; k < NF; ++k) f[k] = 0.0f;
                }
                uint8_t *rowp = myA + lr * 128;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    uint4 w = make_uint4(0u, 0u, 0u, 0u);
                    if (u * 8 < NF)
                        w = make_uint4(pack2(f[8 * u], f[8 * u + 1]), pack2(f[8 * u + 2], f[8 * u + 3]),
                                       pack2(f[8 * u + 4], f[8 * u + 5]), pack2(f[8 * u + 6], f[8 * u + 7]));
                    *(uint4 *)(rowp + ((u ^ (lr & 7)) << 4)) = w;
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            mbar_arrive(&aready);
            for (int l = 0; l < a.n_layers; ++l) {
                if (!mbar_wait(&done, dphase, a.status)) { s_abort = 1; break; }
                dphase ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const float *bias = a.master + a.boff[l];
                if (l + 1 < a.n_layers) {
                    // bias + ReLU -> BF16 -> the next layer's A operand (in place:
                    // every MMA reading it has completed)
#pragma unroll 1
                    for (int c0 = 0; c0 < WID; c0 += 64) {
                        uint32_t r[64];
                        tmem_ld32_nw(trow + (uint32_t)c0, r);
                        tmem_ld32_nw(trow + (uint32_t)(c0 + 32), r + 32);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        uint8_t *rowp = myA + (c0 >> 6) * F_CHUNK + lr * 128;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 b0 = __ldg(reinterpret_cast<const float4 *>(bias + c0 + 8 * q));
                            const float4 b1 = __ldg(reinterpret_cast<const float4 *>(bias + c0 + 8 * q + 4));
                            const float v0 = fmaxf(__uint_as_float(r[8 * q]) + b0.x, 0.0f);
                            const float v1 = fmaxf(__uint_as_float(r[8 * q + 1]) + b0.y, 0.0f);
                            const float v2 = fmaxf(__uint_as_float(r[8 * q + 2]) + b0.z, 0.0f);
                            const float v3 = fmaxf(__uint_as_float(r[8 * q + 3]) + b0.w, 0.0f);
                            const float v4 = fmaxf(__uint_as_float(r[8 * q + 4]) + b1.x, 0.0f);
                            const float v5 = fmaxf(__uint_as_float(r[8 * q + 5]) + b1.y, 0.0f);
                            const float v6 = fmaxf(__uint_as_float(r[8 * q + 6]) + b1.z, 0.0f);
                            const float v7 = fmaxf(__uint_as_float(r[8 * q + 7]) + b1.w, 0.0f);
                            *(uint4 *)(rowp + ((q ^ (lr & 7)) << 4)) =
                                make_uint4(pack2(v0, v1), pack2(v2, v3), pack2(v4, v5), pack2(v6, v7));
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;");
                    mbar_arrive(&aready);
                } else {
                    // head: two linear outputs, de-standardised
                    uint32_t r[32];
                    tmem_ld32_nw(trow, r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    if (row < a.rows) {
                        const float y0 = (__uint_as_float(r[0]) + bias[0]) * s_norm[2 * NF + NO] + s_norm[2 * NF];
                        const float y1 =
                            (__uint_as_float(r[1]) + bias[1]) * s_norm[2 * NF + NO + 1] + s_norm[2 * NF + 1];
                        *reinterpret_cast<float2 *>(a.y + row * NO) = make_float2(y0, y1);
                    }
                    // the next pair's layer-0 arrival (after its input is
                    // written) also releases this TMEM read
                    asm volatile("tcgen05.fence::before_thread_sync;");
                }
            }
        }
    }
    if (tid == 0 && s_abort) atomicOr(&a.status[kStTimeout], 1);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// Training helpers
// ---------------------------------------------------------------------------
// standardised batch: X [R x 64] and X^T [64 x R] (BF16, zero padding), T_s [R x 2]
__global__ void k_prep(const float *x, const float *t, const int32_t *idx, int64_t first, int rows, int R,
                       const float *norm, bf16 *X, bf16 *XT, float *Ts) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= R) return;
    float f[64];
#pragma unroll
    for (int k = 0; k < 64; ++k) f[k] = 0.0f;
    float t0 = 0.0f, t1 = 0.0f;
    if (i < rows) {
        const int64_t src = idx ? (int64_t)idx[first + i] : first + i;
#pragma unroll
        for (int k = 0; k < NF; ++k) f[k] = (x[src * NF + k] - norm[k]) / norm[NF + k];
        t0 = (t[src * NO] - norm[2 * NF]) / norm[2 * NF + NO];
        t1 = (t[src * NO + 1] - norm[2 * NF + 1]) / norm[2 * NF + NO + 1];
    }
#pragma unroll
    for (int k = 0; k < 64; k += 2) *reinterpret_cast<uint32_t *>(X + (int64_t)i * 64 + k) = pack2(f[k], f[k + 1]);
#pragma unroll
    for (int k = 0; k < 64; ++k) XT[(int64_t)k * R + i] = __float2bfloat16(f[k]);
    Ts[2 * i] = t0;
    Ts[2 * i + 1] = t1;
}

// loss and the head's output gradient dZ = (y - t) / rows (zero on padding
// rows), in FP32 [R x 2], BF16 [R x 64] (zero beyond column 1) and BF16 [2 x R];
// one CTA, fixed summation order
__global__ void __launch_bounds__(1024) k_loss(const float *Y, const float *Ts, int rows, int R, float *dZf, bf16 *dZb,
                                               bf16 *dZT, float *loss, float *loss_acc, float acc_w) {
    __shared__ double sh[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) {
        float d0 = 0.0f, d1 = 0.0f;
        if (i < rows) {
            const float e0 = Y[(int64_t)i * 16] - Ts[2 * i], e1 = Y[(int64_t)i * 16 + 1] - Ts[2 * i + 1];
            acc += (double)e0 * e0 + (double)e1 * e1;
            d0 = e0 / (float)rows;
            d1 = e1 / (float)rows;
        }
        dZf[2 * i] = d0;
        dZf[2 * i + 1] = d1;
        uint32_t *zb = reinterpret_cast<uint32_t *>(dZb + (int64_t)i * 64);
        zb[0] = pack2(d0, d1);
        for (int k = 1; k < 32; ++k) zb[k] = 0u;
        dZT[i] = __float2bfloat16(d0);
        dZT[R + i] = __float2bfloat16(d1);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        const float L = (float)(0.5 * s / rows);
        if (loss) *loss = L;
        if (loss_acc) *loss_acc += acc_w * L;
    }
}

// out[c] = sum_r G[r][c] in row order
__global__ void k_colsum(const float *G, int R, int cols, float *out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.0f;
    for (int r = 0; r < R; ++r) s += G[(int64_t)r * cols + c];
    out[c] = s;
}

// Adam on one layer's FP32 parameters (W [out x kin] then b [out]), then the
// BF16 copies: Wf [nout_pad x kin] (forward operand) and Wt [in x kout]
// (backward operand, transposed)
__global__ void k_adam_layer(float *P, const float *G, float *m, float *v, int out, int in, int kin, int kout,
                             float lr, float b1, float b2, float eps, float c1, float c2, int update, bf16 *Wf,
                             bf16 *Wt) {
    const int n = out * kin + out;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float p = P[i];
    if (update) {
        const float g = G[i];
        const float mi = b1 * m[i] + (1.0f - b1) * g;
        const float vi = b2 * v[i] + (1.0f - b2) * g * g;
        m[i] = mi;
        v[i] = vi;
        p -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        P[i] = p;
    }
    if (i < out * kin) {
        const int o = i / kin, k = i % kin;
        Wf[i] = __float2bfloat16(p);
        if (Wt && k < in) Wt[(int64_t)k * kout + o] = __float2bfloat16(p);
    }
}

// the inference image of one layer: chunks (half h, K chunk kc) of
// rows_c x 64 BF16 in the swizzled layout
__global__ void k_pack_img(const float *W, int out, int kin, int rows_c, int n_half, uint8_t *img) {
    const int n_kc = kin / 64;
    const int64_t units = (int64_t)n_half * n_kc * rows_c * 8;
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= units) return;
    const int u = (int)(q & 7);
    const int64_t rest = q >> 3;
    const int n = (int)(rest % rows_c);
    const int chunk = (int)(rest / rows_c);          // h * n_kc + kc
    const int h = chunk / n_kc, kc = chunk % n_kc;
    const int o = h * 128 + n;
    uint32_t w[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int k = kc * 64 + u * 8 + 2 * e;
        const float a0 = o < out ? W[(int64_t)o * kin + k] : 0.0f;
        const float a1 = o < out ? W[(int64_t)o * kin + k + 1] : 0.0f;
        w[e] = pack2(a0, a1);
    }
    *(uint4 *)(img + (int64_t)chunk * rows_c * 128 + n * 128 + ((u ^ (n & 7)) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
}

// ---------------------------------------------------------------------------
// Standalone GEMM status word (the primitive has no network to hold one)
// ---------------------------------------------------------------------------
__device__ int32_t g_gemm_status[4];
std::mutex g_gemm_mu;

}  // namespace

// ---------------------------------------------------------------------------
// Network object
// ---------------------------------------------------------------------------
struct ems_mlp {
    cudaStream_t st = nullptr;
    std::string err;
    int L = 0;                                   // layers (hidden + head)
    int in[MAXL], out[MAXL], kin[MAXL], kout[MAXL], nfwd[MAXL];
    int64_t woff[MAXL], boff[MAXL], n_flat = 0, n_host = 0;
    float *P = nullptr, *G = nullptr, *m = nullptr, *v = nullptr, *norm = nullptr;
    bf16 *Wf[MAXL] = {}, *Wt[MAXL] = {};
    uint8_t *img = nullptr;
    int64_t img_bytes = 0;
    std::vector<int> chunk_off, chunk_info;
    bool img_dirty = true;
    int adam_t = 0;
    int32_t *status = nullptr;
    float *dloss = nullptr;                      // [1] last loss, then per-epoch sums
    int R = 0;                                   // activation capacity (rows)
    bf16 *X = nullptr, *XT = nullptr, *H[MAXL] = {}, *HT[MAXL] = {}, *dZb[2] = {}, *dZT[2] = {};
    float *Ts = nullptr, *Y = nullptr, *dZf[2] = {};
    int32_t *idx = nullptr;
    int64_t idx_cap = 0;
    std::vector<void *> act;                     // activation allocations
};

namespace {

ems_status mfail(ems_mlp *m, ems_status s, const std::string &msg) {
    if (m) m->err = msg;
    return s;
}
ems_status mcuda(ems_mlp *m, cudaError_t e, const char *what) {
    cudaGetLastError();
    return mfail(m, EMS_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}
#define MLP_CUDA(m, call)                                  \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return mcuda((m), e_, #call); \
    } while (0)

ems_status mlp_check_status(ems_mlp *m) {
    int32_t s[4];
    MLP_CUDA(m, cudaMemcpyAsync(s, m->status, sizeof s, cudaMemcpyDeviceToHost, m->st));
    MLP_CUDA(m, cudaStreamSynchronize(m->st));
    if (s[kStTimeout]) {
        cudaMemsetAsync(m->status, 0, sizeof s, m->st);
        return mfail(m, EMS_E_TIMEOUT, "tensor-core kernel: an mbarrier wait ran out its iteration limit");
    }
    return EMS_OK;
}

void free_act(ems_mlp *m) {
    for (void *p : m->act) cudaFree(p);
    m->act.clear();
    m->R = 0;
}

ems_status ensure_act(ems_mlp *m, int R) {
    if (R <= m->R) return EMS_OK;
    free_act(m);
    auto get = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
        m->act.push_back(*p);
        return cudaMemsetAsync(*p, 0, bytes, m->st) == cudaSuccess;
    };
    bool ok = get((void **)&m->X, (size_t)R * 64 * 2) && get((void **)&m->XT, (size_t)R * 64 * 2) &&
              get((void **)&m->Ts, (size_t)R * 2 * 4) && get((void **)&m->Y, (size_t)R * 16 * 4);
    for (int l = 0; ok && l + 1 < m->L; ++l)
        ok = get((void **)&m->H[l], (size_t)R * WID * 2) && get((void **)&m->HT[l], (size_t)R * WID * 2);
    for (int q = 0; ok && q < 2; ++q)
        ok = get((void **)&m->dZf[q], (size_t)R * WID * 4) && get((void **)&m->dZb[q], (size_t)R * WID * 2) &&
             get((void **)&m->dZT[q], (size_t)R * WID * 2);
    if (!ok) { free_act(m); return mfail(m, EMS_E_NOMEM, "activation buffers"); }
    m->R = R;
    return EMS_OK;
}

// BF16 copies (and Adam when update) for every layer
ems_status refresh(ems_mlp *m, bool update, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float c1 = 1.0f, c2 = 1.0f;
    if (update) {
        ++m->adam_t;
        c1 = (float)(1.0 - std::pow(0.9, m->adam_t));
        c2 = (float)(1.0 - std::pow(0.999, m->adam_t));
    }
    for (int l = 0; l < m->L; ++l) {
        const int n = m->out[l] * m->kin[l] + m->out[l];
        k_adam_layer<<<(n + 255) / 256, 256, 0, m->st>>>(m->P + m->woff[l], m->G + m->woff[l], m->m + m->woff[l],
                                                         m->v + m->woff[l], m->out[l], m->in[l], m->kin[l],
                                                         m->kout[l], lr, b1, b2, eps, c1, c2, update ? 1 : 0,
                                                         m->Wf[l], l > 0 ? m->Wt[l] : nullptr);
        MLP_CUDA(m, cudaGetLastError());
    }
    m->img_dirty = true;
    return EMS_OK;
}

GemmArgs gargs(ems_mlp *m, const bf16 *A, const bf16 *B, int M, int N, int K) {
    GemmArgs g{};
    g.A = A; g.B = B; g.M = M; g.N = N; g.K = K; g.scale = 1.0f; g.status = m->status;
    return g;
}

// forward + backward of one batch already prepared in X / XT / Ts (R rows,
// `rows` valid); gradients into m->G, loss into m->dloss[0] (+ acc)
ems_status fwd_bwd(ems_mlp *m, int rows, int R, float *loss_acc, float acc_w) {
    const int L = m->L;
    const bf16 *Hin = m->X;
    for (int l = 0; l < L; ++l) {
        GemmArgs g = gargs(m, Hin, m->Wf[l], R, m->nfwd[l], m->kin[l]);
        g.bias = m->P + m->boff[l];
        if (l + 1 < L) {
            g.relu = 1; g.out_bf16 = m->H[l]; g.out_t = m->HT[l]; g.ldt = R;
            Hin = m->H[l];
        } else {
            g.out_f32 = m->Y;
        }
        MLP_CUDA(m, launch_gemm(m->st, g));
    }
    k_loss<<<1, 1024, 0, m->st>>>(m->Y, m->Ts, rows, R, m->dZf[0], m->dZb[0], m->dZT[0], m->dloss, loss_acc, acc_w);
    MLP_CUDA(m, cudaGetLastError());
    int q = 0;
    for (int l = L - 1; l >= 0; --l) {
        const bf16 *HinT = l == 0 ? m->XT : m->HT[l - 1];
        GemmArgs gw = gargs(m, m->dZT[q], HinT, m->out[l], m->kin[l], R);
        gw.out_f32 = m->G + m->woff[l];
        MLP_CUDA(m, launch_gemm(m->st, gw));
        k_colsum<<<(m->out[l] + 127) / 128, 128, 0, m->st>>>(m->dZf[q], R, m->out[l], m->G + m->boff[l]);
        MLP_CUDA(m, cudaGetLastError());
        if (l > 0) {
            GemmArgs gh = gargs(m, m->dZb[q], m->Wt[l], R, m->in[l], m->kout[l]);
            gh.mask = m->H[l - 1];
            gh.out_f32 = m->dZf[q ^ 1]; gh.out_bf16 = m->dZb[q ^ 1]; gh.out_t = m->dZT[q ^ 1]; gh.ldt = R;
            MLP_CUDA(m, launch_gemm(m->st, gh));
            q ^= 1;
        }
    }
    return EMS_OK;
}

ems_status prep(ems_mlp *m, const float *x, const float *t, const int32_t *idx, int64_t first, int rows, int R) {
    k_prep<<<(R + 127) / 128, 128, 0, m->st>>>(x, t, idx, first, rows, R, m->norm, m->X, m->XT, m->Ts);
    MLP_CUDA(m, cudaGetLastError());
    return EMS_OK;
}

ems_status build_image(ems_mlp *m) {
    if (!m->img_dirty) return EMS_OK;
    int64_t off = 0;
    for (int l = 0; l < m->L; ++l) {
        const int rows_c = m->out[l] >= 128 ? 128 : ((m->out[l] + 15) & ~15);
        const int n_half = (m->out[l] + 127) / 128;
        const int64_t units = (int64_t)n_half * (m->kin[l] / 64) * rows_c * 8;
        k_pack_img<<<(unsigned)((units + 255) / 256), 256, 0, m->st>>>(m->P + m->woff[l], m->out[l], m->kin[l], rows_c,
                                                                      n_half, m->img + off);
        MLP_CUDA(m, cudaGetLastError());
        off += (int64_t)n_half * (m->kin[l] / 64) * rows_c * 128;
    }
    m->img_dirty = false;
    return EMS_OK;
}

void he_init(ems_mlp *m, uint64_t seed, std::vector<float> &host) {
    std::mt19937_64 gen(seed);
    host.assign((size_t)m->n_host, 0.0f);
    size_t o = 0;
    for (int l = 0; l < m->L; ++l) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / m->in[l]));
        for (int i = 0; i < m->out[l] * m->in[l]; ++i) host[o++] = (float)nd(gen);
        o += m->out[l];
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" const char *ems_mlp_last_error(const ems_mlp *m) { return m ? m->err.c_str() : "null network"; }

extern "C" void ems_mlp_destroy(ems_mlp *m) {
    if (!m) return;
    if (m->st) cudaStreamSynchronize(m->st);
    free_act(m);
    for (void *p : {(void *)m->P, (void *)m->G, (void *)m->m, (void *)m->v, (void *)m->norm, (void *)m->img,
                    (void *)m->status, (void *)m->dloss, (void *)m->idx})
        if (p) cudaFree(p);
    for (int l = 0; l < MAXL; ++l) {
        if (m->Wf[l]) cudaFree(m->Wf[l]);
        if (m->Wt[l]) cudaFree(m->Wt[l]);
    }
    delete m;
}

extern "C" ems_status ems_mlp_create(int n_hidden, uint64_t seed, void *stream, ems_mlp **out) {
    if (!out) return EMS_E_INVAL;
    *out = nullptr;
    if (n_hidden < 1 || n_hidden > MAXL - 1) return EMS_E_INVAL;
    ems_mlp *m = new ems_mlp();
    m->st = (cudaStream_t)stream;
    m->L = n_hidden + 1;
    int64_t flat = 0, host = 0, img = 0;
    for (int l = 0; l < m->L; ++l) {
        m->in[l] = l == 0 ? NF : WID;
        m->out[l] = l + 1 == m->L ? NO : WID;
        m->kin[l] = (m->in[l] + 63) / 64 * 64;
        m->kout[l] = (m->out[l] + 63) / 64 * 64;
        m->nfwd[l] = (m->out[l] + 15) / 16 * 16;
        m->woff[l] = flat;
        m->boff[l] = flat + (int64_t)m->out[l] * m->kin[l];
        flat = m->boff[l] + m->out[l];
        flat = (flat + 3) / 4 * 4;                   // 16-byte aligned layers
        host += (int64_t)m->out[l] * m->in[l] + m->out[l];
        const int rows_c = m->out[l] >= 128 ? 128 : ((m->out[l] + 15) & ~15);
        const int n_half = (m->out[l] + 127) / 128;
        for (int h = 0; h < n_half; ++h)
            for (int kc = 0; kc < m->kin[l] / 64; ++kc) {
                m->chunk_off.push_back((int)img);
                m->chunk_info.push_back(l << 16 | h << 8 | kc);
                img += (int64_t)rows_c * 128;
            }
    }
    m->n_flat = flat;
    m->n_host = host;
    m->img_bytes = img;
    auto al = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); return false; }
        return cudaMemsetAsync(*p, 0, bytes, m->st) == cudaSuccess;
    };
    bool ok = al((void **)&m->P, 4 * flat) && al((void **)&m->G, 4 * flat) && al((void **)&m->m, 4 * flat) &&
              al((void **)&m->v, 4 * flat) && al((void **)&m->norm, 4 * (2 * NF + 2 * NO)) &&
              al((void **)&m->img, (size_t)img) && al((void **)&m->status, 16) && al((void **)&m->dloss, 4 * 2048);
    for (int l = 0; ok && l < m->L; ++l) {
        ok = al((void **)&m->Wf[l], (size_t)m->nfwd[l] * m->kin[l] * 2);
        if (ok && l > 0) ok = al((void **)&m->Wt[l], (size_t)m->in[l] * m->kout[l] * 2);
    }
    if (!ok) { ems_mlp_destroy(m); return EMS_E_NOMEM; }
    std::vector<float> nrm(2 * NF + 2 * NO, 0.0f);
    for (int k = 0; k < NF; ++k) nrm[NF + k] = 1.0f;
    nrm[2 * NF + NO] = nrm[2 * NF + NO + 1] = 1.0f;
    if (cudaMemcpyAsync(m->norm, nrm.data(), 4 * nrm.size(), cudaMemcpyHostToDevice, m->st) != cudaSuccess) {
        ems_mlp_destroy(m);
        return EMS_E_CUDA;
    }
    std::vector<float> h;
    he_init(m, seed, h);
    const ems_status s = ems_mlp_set_params(m, h.data());
    if (s != EMS_OK) { ems_mlp_destroy(m); return s; }
    *out = m;
    return EMS_OK;
}

extern "C" int64_t ems_mlp_param_count(const ems_mlp *m) { return m ? m->n_host : 0; }

extern "C" ems_status ems_mlp_set_params(ems_mlp *m, const float *hp) {
    if (!m || !hp) return EMS_E_INVAL;
    std::vector<float> flat((size_t)m->n_flat, 0.0f);
    size_t o = 0;
    for (int l = 0; l < m->L; ++l) {
        for (int r = 0; r < m->out[l]; ++r)
            for (int k = 0; k < m->in[l]; ++k) flat[m->woff[l] + (int64_t)r * m->kin[l] + k] = hp[o++];
        for (int r = 0; r < m->out[l]; ++r) flat[m->boff[l] + r] = hp[o++];
    }
    MLP_CUDA(m, cudaMemcpyAsync(m->P, flat.data(), 4 * flat.size(), cudaMemcpyHostToDevice, m->st));
    MLP_CUDA(m, cudaMemsetAsync(m->m, 0, 4 * m->n_flat, m->st));
    MLP_CUDA(m, cudaMemsetAsync(m->v, 0, 4 * m->n_flat, m->st));
    m->adam_t = 0;
    EMS_TRY(refresh(m, false, 0.0f));
    MLP_CUDA(m, cudaStreamSynchronize(m->st));
    return EMS_OK;
}

static ems_status unpad(ems_mlp *m, const float *dev, float *hp) {
    std::vector<float> flat((size_t)m->n_flat);
    MLP_CUDA(m, cudaMemcpyAsync(flat.data(), dev, 4 * flat.size(), cudaMemcpyDeviceToHost, m->st));
    MLP_CUDA(m, cudaStreamSynchronize(m->st));
    size_t o = 0;
    for (int l = 0; l < m->L; ++l) {
        for (int r = 0; r < m->out[l]; ++r)
            for (int k = 0; k < m->in[l]; ++k) hp[o++] = flat[m->woff[l] + (int64_t)r * m->kin[l] + k];
        for (int r = 0; r < m->out[l]; ++r) hp[o++] = flat[m->boff[l] + r];
    }
    return EMS_OK;
}

extern "C" ems_status ems_mlp_get_params(ems_mlp *m, float *hp) {
    if (!m || !hp) return EMS_E_INVAL;
    return unpad(m, m->P, hp);
}

extern "C" ems_status ems_mlp_set_norm(ems_mlp *m, const float *xm, const float *xs, const float *tm, const float *ts) {
    if (!m || !xm || !xs || !tm || !ts) return EMS_E_INVAL;
    std::vector<float> nrm(2 * NF + 2 * NO);
    for (int k = 0; k < NF; ++k) {
        if (!(xs[k] > 0.0f) || !std::isfinite(xm[k])) return mfail(m, EMS_E_INVAL, "feature std must be > 0");
        nrm[k] = xm[k];
        nrm[NF + k] = xs[k];
    }
    for (int k = 0; k < NO; ++k) {
        if (!(ts[k] > 0.0f) || !std::isfinite(tm[k])) return mfail(m, EMS_E_INVAL, "target std must be > 0");
        nrm[2 * NF + k] = tm[k];
        nrm[2 * NF + NO + k] = ts[k];
    }
    MLP_CUDA(m, cudaMemcpyAsync(m->norm, nrm.data(), 4 * nrm.size(), cudaMemcpyHostToDevice, m->st));
    MLP_CUDA(m, cudaStreamSynchronize(m->st));
    return EMS_OK;
}

namespace {
// Column statistics of a record set for the standardisation: one CTA per
// column (24 feature columns, then 2 target columns), FP64 sums in a fixed
// order (strided per thread, then the block tree), mean first, then the
// centred second moment; std = sqrt(mean square deviation), 1 where it is
// under 1e-6 (a constant column).  Output: x mean, x std, t mean, t std.
__global__ void __launch_bounds__(256) k_col_stats(const float *x, const float *t, int64_t rows, float *norm,
                                                   double *stats) {
    __shared__ double sh[256];
    const int col = blockIdx.x;
    const float *src = col < NF ? x : t;
    const int ld = col < NF ? NF : NO, cc = col < NF ? col : col - NF;
    auto bsum = [&](double v) {
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        const double r = sh[0];
        __syncthreads();
        return r;
    };
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) a += (double)src[i * ld + cc];
    const double mean = bsum(a) / (double)rows;
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < rows; i += blockDim.x) {
        const double d = (double)src[i * ld + cc] - mean;
        q += d * d;
    }
    double sd = sqrt(bsum(q) / (double)rows);
    if (!(sd > 1e-6)) sd = 1.0;
    if (threadIdx.x == 0) {
        const int mo = col < NF ? cc : 2 * NF + cc, so = col < NF ? NF + cc : 2 * NF + NO + cc;
        norm[mo] = (float)mean;
        norm[so] = (float)sd;
        stats[mo] = mean;
        stats[so] = sd;
    }
}
}  // namespace

extern "C" ems_status ems_mlp_fit_norm(ems_mlp *m, const float *x, const float *t, int64_t rows, double *stats) {
    if (!m || !x || !t || rows < 1) return EMS_E_INVAL;
    double *dst = nullptr;
    MLP_CUDA(m, cudaMallocAsync((void **)&dst, sizeof(double) * (2 * NF + 2 * NO), m->st));
    k_col_stats<<<NF + NO, 256, 0, m->st>>>(x, t, rows, m->norm, dst);
    cudaError_t e = cudaGetLastError();
    double h[2 * NF + 2 * NO];
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, dst, sizeof h, cudaMemcpyDeviceToHost, m->st);
    cudaFreeAsync(dst, m->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(m->st);
    if (e != cudaSuccess) return mcuda(m, e, "ems_mlp_fit_norm");
    if (stats)
        for (int k = 0; k < 2 * NF + 2 * NO; ++k) stats[k] = h[k];
    return EMS_OK;
}

extern "C" ems_status ems_mlp_gradients(ems_mlp *m, const float *x, const float *t, int rows, float *grads,
                                        float *loss) {
    if (!m || !x || !t || !grads || rows < 1 || rows > 65536) return EMS_E_INVAL;
    const int R = (rows + 63) / 64 * 64;
    EMS_TRY(ensure_act(m, R));
    EMS_TRY(prep(m, x, t, nullptr, 0, rows, R));
    EMS_TRY(fwd_bwd(m, rows, R, nullptr, 0.0f));
    EMS_TRY(mlp_check_status(m));
    if (loss) MLP_CUDA(m, cudaMemcpy(loss, m->dloss, 4, cudaMemcpyDeviceToHost));
    return unpad(m, m->G, grads);
}

extern "C" ems_status ems_mlp_train_step(ems_mlp *m, const float *x, const float *t, int rows, float lr, float *loss) {
    if (!m || !x || !t || rows < 1 || rows > 65536 || !(lr > 0.0f)) return EMS_E_INVAL;
    const int R = (rows + 63) / 64 * 64;
    EMS_TRY(ensure_act(m, R));
    EMS_TRY(prep(m, x, t, nullptr, 0, rows, R));
    EMS_TRY(fwd_bwd(m, rows, R, nullptr, 0.0f));
    EMS_TRY(refresh(m, true, lr));
    EMS_TRY(mlp_check_status(m));
    if (loss) MLP_CUDA(m, cudaMemcpy(loss, m->dloss, 4, cudaMemcpyDeviceToHost));
    return EMS_OK;
}

extern "C" ems_status ems_mlp_train(ems_mlp *m, const float *x, const float *t, int64_t rows, int batch, int epochs,
                                    float lr, uint64_t seed, float *loss_per_epoch) {
    if (!m || !x || !t || rows < 1 || rows > INT32_MAX || batch < 64 || batch % 64 || batch > 65536 || epochs < 1 ||
        epochs > 1024 || !(lr > 0.0f))
        return EMS_E_INVAL;
    if (rows < batch) return mfail(m, EMS_E_INVAL, "fewer records than one batch");
    EMS_TRY(ensure_act(m, batch));
    if (m->idx_cap < rows) {
        if (m->idx) cudaFree(m->idx);
        m->idx = nullptr;
        if (cudaMalloc(&m->idx, 4 * rows) != cudaSuccess) { cudaGetLastError(); m->idx_cap = 0; return mfail(m, EMS_E_NOMEM, "shuffle index"); }
        m->idx_cap = rows;
    }
    MLP_CUDA(m, cudaMemsetAsync(m->dloss, 0, 4 * 2048, m->st));
    std::vector<int32_t> perm((size_t)rows);
    std::mt19937_64 gen(seed);
    const int64_t nb = rows / batch;
    for (int e = 0; e < epochs; ++e) {
        std::iota(perm.begin(), perm.end(), 0);
        std::shuffle(perm.begin(), perm.end(), gen);
        MLP_CUDA(m, cudaMemcpyAsync(m->idx, perm.data(), 4 * perm.size(), cudaMemcpyHostToDevice, m->st));
        for (int64_t b = 0; b < nb; ++b) {
            EMS_TRY(prep(m, x, t, m->idx, b * batch, batch, batch));
            EMS_TRY(fwd_bwd(m, batch, batch, m->dloss + 1 + e, 1.0f / (float)nb));
            EMS_TRY(refresh(m, true, lr));
        }
        // perm is reused by the next epoch's shuffle: wait for the upload
        MLP_CUDA(m, cudaStreamSynchronize(m->st));
    }
    EMS_TRY(mlp_check_status(m));
    if (loss_per_epoch) MLP_CUDA(m, cudaMemcpy(loss_per_epoch, m->dloss + 1, 4 * epochs, cudaMemcpyDeviceToHost));
    return EMS_OK;
}

namespace ems {
ems_status mlp_sync_status(ems_mlp *m) { return mlp_check_status(m); }
cudaStream_t mlp_stream(const ems_mlp *m) { return m->st; }

ems_status mlp_predict_async(ems_mlp *m, const float *x, int64_t rows, float *y, int64_t *launches) {
    if (rows == 0) return EMS_OK;
    EMS_TRY(build_image(m));
    FusedArgs a{};
    a.x = x; a.y = y; a.rows = rows; a.n_layers = m->L; a.n_chunks = (int)m->chunk_off.size();
    a.img = m->img; a.master = m->P; a.norm = m->norm; a.status = m->status;
    if (a.n_chunks > F_MAXCH) return mfail(m, EMS_E_INVAL, "too many weight chunks");
    for (int l = 0; l < m->L; ++l) { a.boff[l] = (int)m->boff[l]; a.nout[l] = m->out[l]; }
    for (int c = 0; c < a.n_chunks; ++c) { a.chunk_off[c] = m->chunk_off[c]; a.chunk_info[c] = m->chunk_info[c]; }
    int dev = 0, nsm = 0;
    MLP_CUDA(m, cudaGetDevice(&dev));
    MLP_CUDA(m, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    MLP_CUDA(m, cudaFuncSetAttribute(k_mlp_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, F_SMEM));
    const int64_t pairs = (rows + F_ROWS - 1) / F_ROWS;
    const unsigned grid = (unsigned)std::min<int64_t>(pairs, nsm);
    k_mlp_fused<<<grid, F_THREADS, F_SMEM, m->st>>>(a);
    MLP_CUDA(m, cudaGetLastError());
    if (launches) ++*launches;
    return EMS_OK;
}
}  // namespace ems

extern "C" ems_status ems_mlp_predict(ems_mlp *m, const float *x, int64_t rows, float *y) {
    if (!m || rows < 0 || (rows > 0 && (!x || !y))) return EMS_E_INVAL;
    if (((uintptr_t)x & 15) || ((uintptr_t)y & 7)) return mfail(m, EMS_E_INVAL, "x must be 16-byte, y 8-byte aligned");
    EMS_TRY(ems::mlp_predict_async(m, x, rows, y, nullptr));
    return mlp_check_status(m);
}

extern "C" ems_status ems_gemm_bf16(const void *A, const void *B, int M, int N, int K, const float *bias, int relu,
                                    float scale, float *d_f32, void *d_bf16, void *stream) {
    if (!A || !B || !gemm_shape_ok(M, N, K)) return EMS_E_INVAL;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15) || ((uintptr_t)d_f32 & 15) || ((uintptr_t)d_bf16 & 15))
        return EMS_E_INVAL;
    std::lock_guard<std::mutex> lk(g_gemm_mu);
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *status = nullptr;
    if (cudaGetSymbolAddress((void **)&status, g_gemm_status) != cudaSuccess) { cudaGetLastError(); return EMS_E_CUDA; }
    if (cudaMemsetAsync(status, 0, 16, st) != cudaSuccess) { cudaGetLastError(); return EMS_E_CUDA; }
    GemmArgs g{};
    g.A = (const bf16 *)A; g.B = (const bf16 *)B; g.M = M; g.N = N; g.K = K; g.bias = bias; g.relu = relu;
    g.scale = scale; g.out_f32 = d_f32; g.out_bf16 = (bf16 *)d_bf16; g.status = status;
    if (launch_gemm(st, g) != cudaSuccess) { cudaGetLastError(); return EMS_E_CUDA; }
    int32_t s[4];
    if (cudaMemcpyAsync(s, status, 16, cudaMemcpyDeviceToHost, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return EMS_E_CUDA;
    }
    return s[kStTimeout] ? EMS_E_TIMEOUT : EMS_OK;
}
