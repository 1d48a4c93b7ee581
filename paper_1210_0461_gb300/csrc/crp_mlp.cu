// Heavy-pair predictor: a 2 -> 64 -> 64 -> 1 ReLU network on the 5th-gen
// tensor cores (tcgen05).  Not in the paper: it picks pairs that get exact
// reserved counters ahead of the per-partition summaries.
//
// Parameters (fp32 master copy, one flat array): W1[64][2], b1[64],
// W2[64][64], b2[64], w3[64], b3.  The two hidden-layer products run as
// tcgen05.mma kind::f16 with bf16 operands staged in shared memory and fp32
// accumulators in TMEM (M = 128 rows per tile, N = 64); the output layer
// (64 -> 1) is a dot product on the CUDA cores.  The backward pass uses three
// more tensor-core products per tile (dH1 = dZ2 W2, [dW2 | gb2] = dZ2^T [H1 | 1],
// [dW1 | gb1] = dZ1^T [X | 1]; the latter two with the batch as the reduction
// dimension, accumulated in TMEM over all tiles of a CTA).
//
// Shared-memory operands use the canonical K-major layout without swizzle:
// core matrices of 8 rows x 16 bytes (8 bf16); core (r/8, k/8) sits at
// (r/8) * SBO + (k/8) * LBO with LBO = 128 bytes, and one K = 16 step of an
// MMA advances the start address by two cores (256 bytes).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "crp_internal.cuh"

namespace crp {
namespace mlp {

constexpr int kH = 64;
constexpr int kOffW1 = 0, kOffB1 = 128, kOffW2 = 192, kOffB2 = 4288, kOffW3 = 4352, kOffB3 = 4416;
constexpr int kNParam = 4417;
constexpr int kTM = 128;
constexpr int kThreads = 128;
constexpr uint32_t kLBO = 128;
constexpr int kErrTimeout = 1;

__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
    // D f32 (bits 4-5 = 1), A bf16 (bits 7-9 = 1), B bf16 (bits 10-12 = 1),
    // both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t kmaj_off(uint32_t r, uint32_t k, uint32_t sbo) {
    return (r >> 3) * sbo + (k >> 3) * kLBO + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor (no swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= 1ull << 46;  // descriptor version for tcgen05
    return d;
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// D[tmem_col..] (+)= A (M=128 x K) * B (N x K)^T, K = 16 * nk; one thread.
// acc = 0 overwrites D, acc = 1 adds to it.
__device__ __forceinline__ void gemm(uint32_t d_tmem, uint32_t a_saddr, uint32_t a_sbo,
                                     uint32_t b_saddr, uint32_t b_sbo, int N, int nk,
                                     uint32_t acc = 0u) {
    const uint32_t id = idesc_bf16_f32(128, N);
    for (int kk = 0; kk < nk; ++kk)
        mma(d_tmem, sdesc(a_saddr + kk * 2 * kLBO, kLBO, a_sbo),
            sdesc(b_saddr + kk * 2 * kLBO, kLBO, b_sbo), id, (kk > 0 || acc) ? 1u : 0u);
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(mbar) : "memory");
}

// Bounded wait on an mbarrier phase; false after ~0.5 s.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void st_bf16(unsigned char *base, uint32_t off, float v) {
    *(__nv_bfloat16 *)(base + off) = __float2bfloat16_rn(v);
}

// Synchronise the CTA around tensor-core work: make generic smem writes
// visible to the async proxy and order tcgen05 operations across the barrier.
__device__ __forceinline__ void cta_sync_tc() {
    fence_async_smem();
    fence_before();
    __syncthreads();
    fence_after();
}

struct Smem {
    // operand tiles (bf16, canonical K-major core-matrix layout)
    alignas(1024) unsigned char A1[128 * 16 * 2];      // X tile      128 x 16 (K padded)
    alignas(1024) unsigned char B1[64 * 16 * 2];       // W1          64 x 16
    alignas(1024) unsigned char B2[64 * 64 * 2];       // W2          64 x 64
    alignas(1024) unsigned char A2[128 * 64 * 2];      // H1 tile     128 x 64
    alignas(1024) unsigned char AdH[128 * 64 * 2];     // dZ2 tile    128 x 64
    alignas(1024) unsigned char AdW2[128 * 128 * 2];   // dZ2^T       64(+64 zero) x 128
    alignas(1024) unsigned char BdW2[80 * 128 * 2];    // [H1 | 1]^T  80 x 128 (row 64: ones)
    alignas(1024) unsigned char BdH[64 * 64 * 2];      // W2^T        64 x 64
    alignas(1024) unsigned char AdW1[128 * 128 * 2];   // dZ1^T       64(+64 zero) x 128
    alignas(1024) unsigned char BdW1[16 * 128 * 2];    // [X | 1]^T   16 x 128 (row 2: ones)
    float b1[64], b2[64], w3[64], b3;
    float gb1[64], gb2[64], gw3[64], gb3, loss;
    alignas(8) unsigned long long mbar;
    uint32_t tmem;
    int err;
};

__device__ void stage_weights(Smem &s, const float *prm, bool backward) {
    const int tid = threadIdx.x;
    for (int x = tid; x < 64 * 16; x += kThreads) {
        const int n = x >> 4, k = x & 15;
        st_bf16(s.B1, kmaj_off(n, k, 256), k < 2 ? prm[kOffW1 + n * 2 + k] : 0.0f);
    }
    for (int x = tid; x < 64 * 64; x += kThreads) {
        const int n = x >> 6, k = x & 63;
        const float w = prm[kOffW2 + n * 64 + k];
        st_bf16(s.B2, kmaj_off(n, k, 1024), w);
        if (backward) st_bf16(s.BdH, kmaj_off(k, n, 1024), w);   // W2^T
    }
    if (tid < 64) {
        s.b1[tid] = prm[kOffB1 + tid];
        s.b2[tid] = prm[kOffB2 + tid];
        s.w3[tid] = prm[kOffW3 + tid];
        s.gb1[tid] = s.gb2[tid] = s.gw3[tid] = 0.f;
    }
    if (tid == 0) {
        s.b3 = prm[kOffB3];
        s.gb3 = 0.f;
        s.loss = 0.f;
        s.err = 0;
    }
    if (backward) {
        // zero rows 64..127 of the transposed-gradient operands and X^T's pad
        for (int x = tid; x < (int)sizeof(s.AdW2) / 4; x += kThreads) {
            ((uint32_t *)s.AdW2)[x] = 0u;
            ((uint32_t *)s.AdW1)[x] = 0u;
        }
        for (int x = tid; x < (int)sizeof(s.BdW1) / 4; x += kThreads) ((uint32_t *)s.BdW1)[x] = 0u;
        for (int x = tid; x < (int)sizeof(s.BdW2) / 4; x += kThreads) ((uint32_t *)s.BdW2)[x] = 0u;
        __syncthreads();
        // ones rows: the bias gradients come out of the weight-gradient products
        for (int m = tid; m < kTM; m += kThreads) {
            st_bf16(s.BdW2, kmaj_off(64, m, 2048), 1.0f);
            st_bf16(s.BdW1, kmaj_off(2, m, 2048), 1.0f);
        }
    }
}

__device__ void setup_tmem_and_barrier(Smem &s, uint32_t ncols) {
    const int warp = threadIdx.x >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(&s.tmem)), "r"(ncols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    cta_sync_tc();
}

__device__ void teardown_tmem(Smem &s, uint32_t ncols) {
    fence_before();
    __syncthreads();
    fence_after();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(s.tmem),
                     "r"(ncols) : "memory");
}

// All threads wait for the last commit; a timeout is recorded, waited out
// once more (bounded) and reported through err.
__device__ __forceinline__ bool wait_mma(Smem &s, uint32_t &phase) {
    bool ok = mbar_wait(smem_u32(&s.mbar), phase);
    if (!ok) {
        atomicOr(&s.err, kErrTimeout);
        mbar_wait(smem_u32(&s.mbar), phase);
    }
    phase ^= 1u;
    fence_after();
    return ok;
}

// ---------------------------------------------------------------------------
// Forward (inference): y for every row of X (n x 2)
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kThreads, 1)
k_mlp_forward(const float *__restrict__ prm, const float *__restrict__ X, float *__restrict__ Y,
              int64_t n, unsigned int *err_out) {
    extern __shared__ __align__(1024) unsigned char raw[];
    Smem &s = *(Smem *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5;
    stage_weights(s, prm, false);
    setup_tmem_and_barrier(s, 128);
    const uint32_t tm = s.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    const int64_t tiles = (n + kTM - 1) / kTM;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t m = t * kTM + tid;
        const bool valid = m < n;
        const float x0 = valid ? X[2 * m] : 0.f, x1 = valid ? X[2 * m + 1] : 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) st_bf16(s.A1, kmaj_off(tid, k, 256), k == 0 ? x0 : (k == 1 ? x1 : 0.f));
        cta_sync_tc();
        if (tid == 0) {
            gemm(tm, smem_u32(s.A1), 256, smem_u32(s.B1), 256, 64, 1);
            commit(smem_u32(&s.mbar));
        }
        if (__syncthreads_or(!wait_mma(s, phase))) break;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(tm + lane_base + c * 16, v);
#pragma unroll
            for (int q = 0; q < 16; ++q)
                st_bf16(s.A2, kmaj_off(tid, c * 16 + q, 1024), fmaxf(v[q] + s.b1[c * 16 + q], 0.f));
        }
        cta_sync_tc();
        if (tid == 0) {
            gemm(tm + 64, smem_u32(s.A2), 1024, smem_u32(s.B2), 1024, 64, 4);
            commit(smem_u32(&s.mbar));
        }
        if (__syncthreads_or(!wait_mma(s, phase))) break;
        float y = s.b3;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(tm + lane_base + 64 + c * 16, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) y = fmaf(fmaxf(v[q] + s.b2[c * 16 + q], 0.f), s.w3[c * 16 + q], y);
        }
        if (valid) Y[m] = y;
        fence_before();
        __syncthreads();
    }
    teardown_tmem(s, 128);
    if (tid == 0 && s.err) atomicOr(err_out, (unsigned)s.err);
}

// ---------------------------------------------------------------------------
// Loss and gradient: grad += d/dtheta sum_m (y_m - t_m)^2 / n_total
// ---------------------------------------------------------------------------

// Sum over the warp of v[jl], where jl = bit1 + 2 bit2 + 4 bit3 + 8 bit4 of
// the lane (a butterfly reduce-scatter of 16 values: 16 shuffles per lane;
// lanes 2i and 2i + 1 end with the same slot).  v is overwritten.
__device__ __forceinline__ float warp_reduce_scatter16(float *v, int lane) {
#pragma unroll
    for (int w = 8, bit = 16; w >= 1; w >>= 1, bit >>= 1) {
        const bool upper = (lane & bit) != 0;
#pragma unroll
        for (int q = 0; q < w; ++q) {
            const float send = upper ? v[q] : v[q + w];
            const float keep = upper ? v[q + w] : v[q];
            v[q] = keep + __shfl_xor_sync(0xffffffffu, send, bit);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

// TMEM columns: Z1 0..63, Z2 64..127, dH1 128..191 (per tile); the weight
// gradients accumulate over all tiles of the CTA: [dW2 | gb2] 256..335 and
// [dW1 | gb1] 384..399 (the ones rows of [H1 | 1]^T and [X | 1]^T give the
// bias gradients).  gw3 and gb3 are reduced across each warp with shuffles and
// held in registers; one atomic per parameter per CTA at the end.
constexpr uint32_t kColZ1 = 0, kColZ2 = 64, kColDH1 = 128, kColDW2 = 256, kColDW1 = 384;

__global__ void __launch_bounds__(kThreads, 1)
k_mlp_grad(const float *__restrict__ prm, const float *__restrict__ X,
           const float *__restrict__ Tg, int64_t n, float inv_total, float *grad, float *loss,
           unsigned int *err_out) {
    extern __shared__ __align__(1024) unsigned char raw[];
    Smem &s = *(Smem *)(((uintptr_t)raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    stage_weights(s, prm, true);
    setup_tmem_and_barrier(s, 512);
    const uint32_t tm = s.tmem;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
    uint32_t phase = 0;
    float acc_w3[4] = {0.f, 0.f, 0.f, 0.f};   // gw3[c * 16 + slot(lane)] of this warp
    float acc_b3 = 0.f, acc_loss = 0.f;        // lane 0 of each warp
    bool first = true, ok = true;
    const int64_t tiles = (n + kTM - 1) / kTM;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        const int64_t m = t * kTM + tid;
        const bool valid = m < n;
        const float x0 = valid ? X[2 * m] : 0.f, x1 = valid ? X[2 * m + 1] : 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) st_bf16(s.A1, kmaj_off(tid, k, 256), k == 0 ? x0 : (k == 1 ? x1 : 0.f));
        st_bf16(s.BdW1, kmaj_off(0, tid, 2048), x0);   // [X | 1]^T rows 0, 1
        st_bf16(s.BdW1, kmaj_off(1, tid, 2048), x1);
        cta_sync_tc();
        if (tid == 0) {
            gemm(tm + kColZ1, smem_u32(s.A1), 256, smem_u32(s.B1), 256, 64, 1);
            commit(smem_u32(&s.mbar));
        }
        if (__syncthreads_or(!wait_mma(s, phase))) { ok = false; break; }
        uint64_t mask1 = 0;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(tm + lane_base + kColZ1 + c * 16, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = c * 16 + q;
                const float z = v[q] + s.b1[j];
                const float h = valid ? fmaxf(z, 0.f) : 0.f;
                if (z > 0.f) mask1 |= 1ull << j;
                st_bf16(s.A2, kmaj_off(tid, j, 1024), h);
                st_bf16(s.BdW2, kmaj_off(j, tid, 2048), h);   // [H1 | 1]^T rows 0..63
            }
        }
        cta_sync_tc();
        if (tid == 0) {
            gemm(tm + kColZ2, smem_u32(s.A2), 1024, smem_u32(s.B2), 1024, 64, 4);
            commit(smem_u32(&s.mbar));
        }
        if (__syncthreads_or(!wait_mma(s, phase))) { ok = false; break; }
        float y = s.b3;
        uint64_t mask2 = 0;
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(tm + lane_base + kColZ2 + c * 16, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = c * 16 + q;
                const float z = v[q] + s.b2[j];
                if (z > 0.f) mask2 |= 1ull << j;
                y = fmaf(fmaxf(z, 0.f), s.w3[j], y);
            }
        }
        const float r = valid ? y - Tg[m] : 0.f;
        const float dy = 2.f * r * inv_total;
        {
            const float l = warp_sum(r * r * inv_total), g = warp_sum(dy);
            if (lane == 0) { acc_loss += l; acc_b3 += g; }
        }
        for (int c = 0; c < 4; ++c) {
            float v[16], gw[16];
            tmem_ld16(tm + lane_base + kColZ2 + c * 16, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = c * 16 + q;
                gw[q] = fmaxf(v[q] + s.b2[j], 0.f) * dy;
                const float dz = ((mask2 >> j) & 1ull) ? dy * s.w3[j] : 0.f;
                st_bf16(s.AdH, kmaj_off(tid, j, 1024), dz);
                st_bf16(s.AdW2, kmaj_off(j, tid, 2048), dz);   // dZ2^T
            }
            acc_w3[c] += warp_reduce_scatter16(gw, lane);
        }
        cta_sync_tc();
        if (tid == 0) {
            gemm(tm + kColDH1, smem_u32(s.AdH), 1024, smem_u32(s.BdH), 1024, 64, 4);     // dH1
            gemm(tm + kColDW2, smem_u32(s.AdW2), 2048, smem_u32(s.BdW2), 2048, 80, 8,
                 first ? 0u : 1u);                                                       // [dW2|gb2]
            commit(smem_u32(&s.mbar));
        }
        if (__syncthreads_or(!wait_mma(s, phase))) { ok = false; break; }
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tmem_ld16(tm + lane_base + kColDH1 + c * 16, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int j = c * 16 + q;
                const float dz1 = ((mask1 >> j) & 1ull) ? v[q] : 0.f;
                st_bf16(s.AdW1, kmaj_off(j, tid, 2048), dz1);   // dZ1^T
            }
        }
        cta_sync_tc();
        if (tid == 0) {
            gemm(tm + kColDW1, smem_u32(s.AdW1), 2048, smem_u32(s.BdW1), 2048, 16, 8,
                 first ? 0u : 1u);                                                       // [dW1|gb1]
            commit(smem_u32(&s.mbar));
        }
        // the next tile's first writes (A1, BdW1, A2, BdW2, AdW1) must wait for
        // this product: every tile ends with a completed MMA
        if (__syncthreads_or(!wait_mma(s, phase))) { ok = false; break; }
        first = false;
    }
    // read the accumulated weight gradients (every warp issues the loads)
    if (ok && !first) {
        for (int c = 0; c < 5; ++c) {
            float v[16];
            tmem_ld16(tm + lane_base + kColDW2 + c * 16, v);
            if (tid < 64) {
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int col = c * 16 + q;
                    if (col < 64) atomicAdd(&grad[kOffW2 + tid * 64 + col], v[q]);
                    else if (col == 64) atomicAdd(&grad[kOffB2 + tid], v[q]);
                }
            }
        }
        float v[16];
        tmem_ld16(tm + lane_base + kColDW1, v);
        if (tid < 64) {
            atomicAdd(&grad[kOffW1 + tid * 2 + 0], v[0]);
            atomicAdd(&grad[kOffW1 + tid * 2 + 1], v[1]);
            atomicAdd(&grad[kOffB1 + tid], v[2]);
        }
        if ((lane & 1) == 0) {
            const int slot = ((lane >> 1) & 1) + 2 * ((lane >> 2) & 1) + 4 * ((lane >> 3) & 1) +
                             8 * ((lane >> 4) & 1);
#pragma unroll
            for (int c = 0; c < 4; ++c) atomicAdd(&grad[kOffW3 + c * 16 + slot], acc_w3[c]);
        }
        if (lane == 0) {
            atomicAdd(&grad[kOffB3], acc_b3);
            atomicAdd(loss, acc_loss);
        }
    }
    teardown_tmem(s, 512);
    if (tid == 0 && s.err) atomicOr(err_out, (unsigned)s.err);
}

// Adam (Kingma & Ba 2015) on the fp32 master parameters.
__global__ void k_adam(float *prm, float *m1, float *m2, const float *g, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const float gg = g[x];
        const float a = b1 * m1[x] + (1.f - b1) * gg;
        const float b = b2 * m2[x] + (1.f - b2) * gg * gg;
        m1[x] = a;
        m2[x] = b;
        prm[x] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
    }
}

size_t smem_bytes() { return sizeof(Smem) + 1024; }

}  // namespace mlp
}  // namespace crp

using namespace crp;

static unsigned int *mlp_err_buffer(int dev) {
    static unsigned int *bufs[64] = {};
    if (dev < 0 || dev >= 64) return nullptr;
    if (!bufs[dev] && cudaMalloc(&bufs[dev], sizeof(unsigned int)) != cudaSuccess) return nullptr;
    return bufs[dev];
}

static crp_status mlp_finish(cudaStream_t s, unsigned int *err, const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
        return CRP_ECUDA;
    }
    unsigned int h = 0;
    e = cudaMemcpyAsync(&h, err, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_last_error(std::string(what) + ": " + cudaGetErrorString(e));
        return CRP_ECUDA;
    }
    if (h & mlp::kErrTimeout) {
        set_last_error(std::string(what) + ": a tensor-core completion wait timed out");
        return CRP_ETIMEOUT;
    }
    return CRP_OK;
}

extern "C" int32_t crp_mlp_param_count(void) { return mlp::kNParam; }

extern "C" crp_status crp_mlp_forward(const float *params, const float *x, float *y, int64_t n,
                                      void *stream) {
    if (!params || n < 0 || (n > 0 && (!x || !y))) {
        set_last_error("crp_mlp_forward: bad argument");
        return CRP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned int *err = mlp_err_buffer(dev);
    if (!err) return CRP_ENOMEM;
    cudaMemsetAsync(err, 0, 4, s);
    if (n == 0) return CRP_OK;
    const size_t smem = mlp::smem_bytes();
    cudaFuncSetAttribute(mlp::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t tiles = (n + mlp::kTM - 1) / mlp::kTM;
    const int grid = (int)(tiles < sms ? tiles : sms);
    mlp::k_mlp_forward<<<grid, mlp::kThreads, smem, s>>>(params, x, y, n, err);
    return mlp_finish(s, err, "crp_mlp_forward");
}

extern "C" crp_status crp_mlp_grad(const float *params, const float *x, const float *t, int64_t n,
                                   int64_t n_total, float *grad, float *loss, void *stream) {
    if (!params || !grad || !loss || n < 0 || (n > 0 && (!x || !t)) || n_total <= 0) {
        set_last_error("crp_mlp_grad: bad argument");
        return CRP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    unsigned int *err = mlp_err_buffer(dev);
    if (!err) return CRP_ENOMEM;
    cudaMemsetAsync(err, 0, 4, s);
    cudaMemsetAsync(grad, 0, mlp::kNParam * sizeof(float), s);
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    if (n == 0) return CRP_OK;
    const size_t smem = mlp::smem_bytes();
    cudaFuncSetAttribute(mlp::k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int64_t tiles = (n + mlp::kTM - 1) / mlp::kTM;
    const int grid = (int)(tiles < sms ? tiles : sms);
    mlp::k_mlp_grad<<<grid, mlp::kThreads, smem, s>>>(params, x, t, n, 1.0f / (float)n_total, grad,
                                                      loss, err);
    return mlp_finish(s, err, "crp_mlp_grad");
}

extern "C" crp_status crp_mlp_adam(float *params, float *m, float *v, const float *grad, float lr,
                                   int32_t step, void *stream) {
    if (!params || !m || !v || !grad || step < 1) {
        set_last_error("crp_mlp_adam: bad argument");
        return CRP_EINVAL;
    }
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    mlp::k_adam<<<(mlp::kNParam + 255) / 256, 256, 0, (cudaStream_t)stream>>>(
        params, m, v, grad, mlp::kNParam, lr, b1, b2, 1e-8f, c1, c2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("crp_mlp_adam: ") + cudaGetErrorString(e));
        return CRP_ECUDA;
    }
    return CRP_OK;
}
