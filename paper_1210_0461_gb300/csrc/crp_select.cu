// Selections on the GPU: item counts over a compressed index array, and the
// indices of the K largest 32-bit keys (MSD radix select, 8-bit digits, ties
// at the threshold taken in arbitrary order).
#include <cuda_runtime.h>
#include <stdint.h>

#include "crp_internal.cuh"

namespace crp {

// Item counts with on-chip combining: each CTA counts into a shared-memory
// table of kCountSlots items (open addressing, a few probes; an item that
// finds no slot is counted straight in global memory) and adds the table into
// cnt at the end, so a frequent item costs one global atomic per CTA rather
// than one per occurrence.  nnz_at, when given, holds the count on the device
// (an entry of a ptr array).
constexpr int kCountSlots = 2048;
constexpr int kCountProbes = 8;
__global__ void __launch_bounds__(256) k_item_counts(const int32_t *idx, int64_t nnz,
                                                     const int64_t *nnz_at, int32_t n_items,
                                                     unsigned int *cnt) {
    __shared__ unsigned int key[kCountSlots], val[kCountSlots];
    for (int t = threadIdx.x; t < kCountSlots; t += blockDim.x) {
        key[t] = 0xFFFFFFFFu;
        val[t] = 0u;
    }
    __syncthreads();
    if (nnz_at) nnz = *nnz_at;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = idx[x];
        if (v < 0 || v >= n_items) continue;
        uint32_t h = ((uint32_t)v * 2654435761u) >> 21;   // 11 bits: kCountSlots
        bool done = false;
        for (int pr = 0; pr < kCountProbes; ++pr, h = (h + 1) & (kCountSlots - 1)) {
            unsigned int k = key[h];
            if (k == 0xFFFFFFFFu) k = atomicCAS(&key[h], 0xFFFFFFFFu, (unsigned int)v);
            if (k == 0xFFFFFFFFu || k == (unsigned int)v) {
                atomicAdd(&val[h], 1u);
                done = true;
                break;
            }
        }
        if (!done) atomicAdd(&cnt[v], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kCountSlots; t += blockDim.x)
        if (val[t]) atomicAdd(&cnt[key[t]], val[t]);
}

// Selection state kept on the device between passes (no host round trip):
// words 258 and 259 of the scratch hold the count still wanted at the
// current prefix and the prefix itself.
constexpr int kSelNeed = 258, kSelPrefix = 259;

__global__ void k_sel_hist(const uint32_t *key, int64_t n, int pass, unsigned int *scratch) {
    __shared__ unsigned int h[256];
    const int shift = 24 - 8 * pass;
    const uint32_t prefix = pass ? scratch[kSelPrefix] : 0u;
    const uint32_t pmask = pass ? 0xFFFFFFFFu << (shift + 8) : 0u;
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = key[x];
        if ((k & pmask) == prefix) atomicAdd(&h[(k >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&scratch[t], h[t]);
}

// The digit of this pass: the largest d whose keys (with the prefix so far)
// together with those of the larger digits reach the wanted count; the
// wanted count drops by the keys of the larger digits. Clears the histogram
// for the next pass. One CTA of 256 threads.
__global__ void k_sel_pick(unsigned int *scratch, int pass, uint32_t K) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = scratch[threadIdx.x];   // one parallel read of the histogram
    __syncthreads();
    if (threadIdx.x == 0) {
        const int shift = 24 - 8 * pass;
        uint32_t need = pass ? scratch[kSelNeed] : K;
        const uint32_t prefix = pass ? scratch[kSelPrefix] : 0u;
        uint64_t cum = 0;
        int d = 255;
        for (; d > 0; --d) {
            if (cum + h[d] >= need) break;
            cum += h[d];
        }
        need -= (uint32_t)cum;
        scratch[kSelNeed] = need;
        scratch[kSelPrefix] = prefix | ((uint32_t)d << shift);
    }
    scratch[threadIdx.x] = 0;   // (every thread read its bin before the barrier)
}

__global__ void k_sel_emit(const uint32_t *key, int64_t n, const unsigned int *scratch,
                           int64_t *out, unsigned int *cnt, unsigned int *tie) {
    const uint32_t tau = scratch[kSelPrefix], need_at_tau = scratch[kSelNeed];
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = key[x];
        bool take = k > tau;
        if (k == tau) take = atomicAdd(tie, 1u) < need_at_tau;
        if (take) out[atomicAdd(cnt, 1u)] = x;
    }
}

// CTAs of the counting kernel: enough for the input, at most 512 (each adds
// its shared-memory table into the counts at the end, so more CTAs would
// only repeat the frequent items' global atomics).
static int count_grid_for(int64_t n) {
    const int64_t g = (n + 4095) / 4096;
    return (int)(g < 512 ? (g > 0 ? g : 1) : 512);
}

int select_grid_for(int64_t n) {
    int64_t g = (n + 255) / 256;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

// Indices (unordered) of the K largest keys.  out: device, K entries.
// Four histogram passes and the emit run back to back on the stream; the
// digits are picked on the device, so the host never waits.
cudaError_t select_top(const uint32_t *key, int64_t n, int64_t K, int64_t *out,
                       unsigned int *scratch /* 260 */, cudaStream_t s) {
    if (K < 0 || K > (int64_t)0xFFFFFFFFu) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 258 * 4, s);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 4; ++pass) {
        k_sel_hist<<<select_grid_for(n), 256, 0, s>>>(key, n, pass, scratch);
        k_sel_pick<<<1, 256, 0, s>>>(scratch, pass, (uint32_t)K);
    }
    k_sel_emit<<<select_grid_for(n), 256, 0, s>>>(key, n, scratch, out, scratch + 256,
                                                  scratch + 257);
    return cudaGetLastError();
}


// Reorder items[0, R) by descending cnt[item] (ties in any order): one CTA,
// bitonic sort of R <= 4096 keys (cnt << 32 | 1 << 31 | item) in shared memory.
__global__ void __launch_bounds__(1024) k_order_by_count(int64_t *items, const unsigned int *cnt,
                                                         uint32_t R) {
    __shared__ unsigned long long key[4096];
    uint32_t n = 1;
    while (n < R) n <<= 1;
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x)
        key[t] = t < R ? ((unsigned long long)cnt[items[t]] << 32) | (1ull << 31) |
                             (unsigned long long)items[t]
                       : 0ull;
    __syncthreads();
    for (uint32_t size = 2; size <= n; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
            for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
                const uint32_t u = t ^ stride;
                if (u > t) {
                    const bool desc = (t & size) == 0;
                    const unsigned long long a = key[t], b = key[u];
                    if (desc ? a < b : a > b) { key[t] = b; key[u] = a; }
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t t = threadIdx.x; t < R; t += blockDim.x)
        items[t] = (int64_t)(key[t] & 0x7FFFFFFFull);
}

cudaError_t order_by_count(int64_t *items, const unsigned int *cnt, uint32_t R, cudaStream_t s) {
    if (R == 0 || R > 4096) return R == 0 ? cudaSuccess : cudaErrorInvalidValue;
    k_order_by_count<<<1, 1024, 0, s>>>(items, cnt, R);
    return cudaGetLastError();
}

cudaError_t launch_item_counts(const int32_t *idx, int64_t nnz, int32_t n_items, unsigned int *cnt,
                               cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    k_item_counts<<<count_grid_for(nnz), 256, 0, s>>>(idx, nnz, nullptr, n_items, cnt);
    return cudaGetLastError();
}

// The same over idx[0, *nnz_at) with the count read on the device (no host
// round trip); nnz_hint sizes the grid only.
cudaError_t launch_item_counts_at(const int32_t *idx, const int64_t *nnz_at, int64_t nnz_hint,
                                  int32_t n_items, unsigned int *cnt, cudaStream_t s) {
    k_item_counts<<<count_grid_for(nnz_hint), 256, 0, s>>>(idx, 0, nnz_at, n_items, cnt);
    return cudaGetLastError();
}

}  // namespace crp
