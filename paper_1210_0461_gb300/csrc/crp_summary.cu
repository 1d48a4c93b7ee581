// Per-partition counter summaries with Space-Saving guarantees
// (Preliminaries, "Frequent items mining algorithms"; Figure 1 updates the
// summary SS[h(e)] of each entry's bucket).
//
// The sequential Space-Saving update (replace the minimum counter) does not
// parallelise, so the GPU keeps each partition's summary as a hash table that
// may hold up to 2*ell keys between compactions:
//   * a recorded key adds its (exact, window-combined) weight;
//   * a new key is recorded as (floor + w, overestimation floor), where the
//     floor bounds the weight of every unrecorded key of the partition;
//   * k_summary_compact keeps the ell keys of largest count, raises the
//     floor to the ell-th largest count and rebuilds the table.
// Between compactions a partition may hold up to 2*ell keys (more counters
// only sharpen the estimates); it is compacted once it holds more than
// 7/4 ell, and every partition is compacted to ell at the end of each call.
// Each compaction drops at least as many keys as were added since the last
// one, each with count >= the old floor, so the sum of kept counts never
// exceeds the partition's stream weight W; hence floor <= W / ell, every
// estimate overshoots by at most W / ell, and every key heavier than W / ell
// is kept -- the guarantees the paper quotes for Space-Saving.
#include <cuda_runtime.h>
#include <stdint.h>

#include "crp_internal.cuh"

namespace crp {

constexpr int kCompactThreads = 1024;

__device__ __forceinline__ unsigned int slot_count(const Slot &s) { return (unsigned int)s.val; }

// One CTA per partition (grid-stride over todo[]).  tmp holds ell slots per CTA.
__global__ void __launch_bounds__(kCompactThreads)
k_summary_compact(Slot *slots, const unsigned long long *part_off,
                  const unsigned long long *part_mask, unsigned int *live, unsigned int *floor,
                  const unsigned int *todo, uint32_t n_todo, uint32_t ell, uint32_t trigger,
                  Slot *tmp) {
    __shared__ unsigned int hist[2048];
    __shared__ unsigned int sel_digit, need_s, kept_n, tie_n;
    Slot *mine = tmp + (size_t)blockIdx.x * ell;
    for (uint32_t t = blockIdx.x; t < n_todo; t += gridDim.x) {
        const uint32_t p = todo ? todo[t] : t;
        if (live[p] <= trigger) continue;
        const unsigned long long off = part_off[p], cap = part_mask[p] + 1ull;
        // radix select of the ell-th largest count: digits of 11, 11, 10 bits
        unsigned int prefix = 0, pmask = 0;
        if (threadIdx.x == 0) need_s = ell;
        const int shifts[3] = {21, 10, 0};
        const unsigned int widths[3] = {11, 11, 10};
        for (int pass = 0; pass < 3; ++pass) {
            const unsigned int dmask = (1u << widths[pass]) - 1u;
            for (int b = threadIdx.x; b < 2048; b += kCompactThreads) hist[b] = 0;
            __syncthreads();
            for (unsigned long long x = threadIdx.x; x < cap; x += kCompactThreads) {
                const Slot s = slots[off + x];
                if (s.key == kEmptyKey) continue;
                const unsigned int c = slot_count(s);
                if ((c & pmask) != prefix) continue;
                atomicAdd(&hist[(c >> shifts[pass]) & dmask], 1u);
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned int cum = 0, need = need_s;
                int d = (int)dmask;
                for (; d > 0; --d) {
                    if (cum + hist[d] >= need) break;
                    cum += hist[d];
                }
                sel_digit = (unsigned int)d;
                need_s = need - cum;
            }
            __syncthreads();
            prefix |= sel_digit << shifts[pass];
            pmask |= dmask << shifts[pass];
        }
        const unsigned int tau = prefix;     // the ell-th largest count
        const unsigned int at_tau = need_s;  // keys at tau that stay
        if (threadIdx.x == 0) { kept_n = 0; tie_n = 0; }
        __syncthreads();
        for (unsigned long long x = threadIdx.x; x < cap; x += kCompactThreads) {
            const Slot s = slots[off + x];
            if (s.key == kEmptyKey) continue;
            const unsigned int c = slot_count(s);
            bool keep = c > tau;
            if (c == tau) keep = atomicAdd(&tie_n, 1u) < at_tau;
            if (keep) mine[atomicAdd(&kept_n, 1u)] = s;
        }
        __syncthreads();
        for (unsigned long long x = threadIdx.x; x < cap; x += kCompactThreads) {
            slots[off + x].key = kEmptyKey;
            slots[off + x].val = 0ull;
        }
        __syncthreads();
        const unsigned long long mask = cap - 1ull;
        const unsigned int n = kept_n;
        for (unsigned int y = threadIdx.x; y < n; y += kCompactThreads) {
            const Slot s = mine[y];
            unsigned long long h = slot_mix(s.key) & mask;
            for (unsigned long long probe = 0; probe <= mask; ++probe) {
                if (atomicCAS(&slots[off + h].key, kEmptyKey, s.key) == kEmptyKey) {
                    slots[off + h].val = s.val;
                    break;
                }
                h = (h + 1) & mask;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            live[p] = n;
            if (tau > floor[p]) floor[p] = tau;
        }
        __syncthreads();
    }
}

cudaError_t launch_summary_compact(Slot *slots, const unsigned long long *part_off,
                                   const unsigned long long *part_mask, unsigned int *live,
                                   unsigned int *floor, const unsigned int *todo, uint32_t n_todo,
                                   uint32_t ell, uint32_t trigger, Slot *tmp, int grid,
                                   cudaStream_t s) {
    if (n_todo == 0) return cudaSuccess;
    k_summary_compact<<<grid, kCompactThreads, 0, s>>>(slots, part_off, part_mask, live, floor,
                                                       todo, n_todo, ell, trigger, tmp);
    return cudaGetLastError();
}

// Reserved exact counters: insert keys (count 0) into the reserved region.
__global__ void k_reserve_insert(Slot *slots, unsigned long long res_off,
                                 unsigned long long res_mask, const unsigned long long *keys,
                                 int32_t n) {
    for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const unsigned long long key = keys[x];
        unsigned long long h = slot_mix(key) & res_mask;
        for (unsigned long long probe = 0; probe <= res_mask; ++probe) {
            const unsigned long long prev = atomicCAS(&slots[res_off + h].key, kEmptyKey, key);
            if (prev == kEmptyKey || prev == key) break;
            h = (h + 1) & res_mask;
        }
    }
}

cudaError_t launch_reserve_insert(Slot *slots, unsigned long long res_off,
                                  unsigned long long res_mask, const unsigned long long *keys,
                                  int32_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_reserve_insert<<<(n + 255) / 256, 256, 0, s>>>(slots, res_off, res_mask, keys, n);
    return cudaGetLastError();
}

// Mark the row and column indices that occur in reserved keys.
__global__ void k_reserve_bits(const unsigned long long *keys, int32_t n, unsigned int *bits_a,
                               unsigned int *bits_b) {
    for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)(keys[x] >> 32), j = (uint32_t)keys[x];
        atomicOr(&bits_a[i >> 5], 1u << (i & 31));
        atomicOr(&bits_b[j >> 5], 1u << (j & 31));
    }
}

cudaError_t launch_reserve_bits(const unsigned long long *keys, int32_t n, unsigned int *bits_a,
                                unsigned int *bits_b, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_reserve_bits<<<(n + 255) / 256, 256, 0, s>>>(keys, n, bits_a, bits_b);
    return cudaGetLastError();
}

}  // namespace crp
