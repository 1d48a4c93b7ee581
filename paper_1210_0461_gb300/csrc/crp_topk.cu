// Heaviest entries of the partition tables (Section 6: the task is to find
// the largest entries of the product) and table export.
//
// crp_topk runs:  (1) a log-linear histogram of the weights, over a 1/32
// sample of the slots for a large table, (2) one pass collecting the slots at
// or above the bucket that the histogram puts at or below the k-th largest
// weight (with a sample, a bucket expected to hold several times k; if fewer
// than k slots come back, the full histogram is taken and the pass redone:
// k collected slots at or above a bucket contain every slot of the top k),
// (3) when that candidate set is still
// larger than one CTA can sort, an MSD radix select over the 128-bit order
// key (weight descending, then (i, j) ascending) on the candidates only, and
// (4) a single-CTA bitonic sort of the k survivors that writes the output.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "crp_internal.cuh"
#include "crp_topk.cuh"

namespace crp {

// Order-preserving 64-bit key of |w|: int counts as they are, doubles by the
// bit pattern of their absolute value (IEEE order equals unsigned order for
// non-negative doubles).
__device__ __forceinline__ unsigned long long weight_key(const Slot &s, int value_type,
                                                         double &w) {
    if (value_type != CRP_F32_COMP) {  // int counts, or summary upper bounds
        unsigned int c = (unsigned int)s.val;
        w = (double)c;
        return c;
    }
    w = __longlong_as_double((long long)s.val);
    return (unsigned long long)__double_as_longlong(fabs(w));
}

// Lower bound of an entry: the weight itself for exact tables, count minus
// overestimation for summary slots (value type kVTSummary).
__device__ __forceinline__ double weight_lower(const Slot &s, int value_type, double w) {
    if (value_type == kVTSummary)
        return (double)((unsigned int)s.val - (unsigned int)(s.val >> 32));
    return w;
}

// 65 exponents x 64 sub-buckets, but capped to kTopkBuckets.
__host__ __device__ __forceinline__ unsigned int bucket_of(unsigned long long u) {
    if (u == 0) return 0;
#ifdef __CUDA_ARCH__
    int e = 63 - __clzll((long long)u);
#else
    int e = 63 - __builtin_clzll(u);
#endif
    unsigned int m = e >= 6 ? (unsigned int)((u >> (e - 6)) & 63u)
                            : (unsigned int)((u << (6 - e)) & 63u);
    unsigned int b = 1u + (unsigned int)e * 64u + m;
    return b < (unsigned)kTopkBuckets ? b : (unsigned)kTopkBuckets - 1u;
}

unsigned int topk_bucket_host(unsigned long long u) { return bucket_of(u); }

// Histogram of the weights of all slots, or (sample_shift = s > 0) of the
// first 32 slots of every 32 << s: a 2^-s sample read in whole 512-byte runs.
__global__ void k_topk_hist(const Slot *__restrict__ slots, uint64_t n, int value_type,
                            int upper_only, int sample_shift, unsigned int *__restrict__ hist) {
    __shared__ unsigned int h[kTopkBuckets];
    for (int t = threadIdx.x; t < kTopkBuckets; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const uint64_t m = sample_shift ? ((n >> 5) >> sample_shift) << 5 : n;
    for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < m;
         y += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = sample_shift ? ((y >> 5) << (5 + sample_shift)) + (y & 31) : y;
        Slot s = slots[x];
        if (s.key == kEmptyKey) continue;
        if (upper_only && !((uint32_t)(s.key >> 32) < (uint32_t)s.key)) continue;
        double w;
        atomicAdd(&h[bucket_of(weight_key(s, value_type, w))], 1u);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kTopkBuckets; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

cudaError_t launch_topk_hist(const Slot *slots, uint64_t n, int value_type, int upper_only,
                             int sample_shift, unsigned int *hist, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * kTopkBuckets, s);
    if (e != cudaSuccess || n == 0) return e;
    uint64_t blocks = ((sample_shift ? n >> sample_shift : n) + 511) / 512;
    int grid = (int)(blocks < 4096 ? (blocks > 0 ? blocks : 1) : 4096);
    k_topk_hist<<<grid, 512, 0, s>>>(slots, n, value_type, upper_only, sample_shift, hist);
    return cudaGetLastError();
}

__global__ void k_topk_collect(const Slot *__restrict__ slots, uint64_t n, int value_type,
                               int upper_only, unsigned int bucket_lo, TopkCand *out,
                               unsigned int *count, unsigned int cap) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        Slot s = slots[x];
        if (s.key == kEmptyKey) continue;
        if (upper_only && !((uint32_t)(s.key >> 32) < (uint32_t)s.key)) continue;
        double w;
        unsigned long long u = weight_key(s, value_type, w);
        if (bucket_of(u) < bucket_lo) continue;
        unsigned int at = atomicAdd(count, 1u);
        if (at < cap) {
            TopkCand c;
            c.wkey = u;
            c.ij = s.key;
            c.w = w;
            c.wl = weight_lower(s, value_type, w);
            out[at] = c;
        }
    }
}

cudaError_t launch_topk_collect(const Slot *slots, uint64_t n, int value_type, int upper_only,
                                unsigned int bucket_lo, TopkCand *out, unsigned int *count,
                                unsigned int cap, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess || n == 0) return e;
    uint64_t blocks = (n + 511) / 512;
    int grid = (int)(blocks < 4096 ? blocks : 4096);
    k_topk_collect<<<grid, 512, 0, s>>>(slots, n, value_type, upper_only, bucket_lo, out, count,
                                        cap);
    return cudaGetLastError();
}

// Digit d (0 = most significant) of the descending 128-bit order key
// Log-linear histogram of candidates' weights (the buckets of the table scan)
// and the candidates at or above a bucket: the first cut of a selection among
// many candidates, before any radix pass.
__global__ void k_cand_hist(const TopkCand *__restrict__ c, unsigned int n, unsigned int *hist) {
    __shared__ unsigned int h[kTopkBuckets];
    for (int t = threadIdx.x; t < kTopkBuckets; t += blockDim.x) h[t] = 0;
    __syncthreads();
    for (unsigned int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        atomicAdd(&h[bucket_of(c[x].wkey)], 1u);
    __syncthreads();
    for (int t = threadIdx.x; t < kTopkBuckets; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

cudaError_t launch_cand_hist(const TopkCand *c, unsigned int n, unsigned int *hist,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * kTopkBuckets, s);
    if (e != cudaSuccess || n == 0) return e;
    unsigned int blocks = (n + 255) / 256;
    k_cand_hist<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(c, n, hist);
    return cudaGetLastError();
}

__global__ void k_cand_collect(const TopkCand *__restrict__ c, unsigned int n, unsigned int b_lo,
                               TopkCand *out, unsigned int *cnt) {
    for (unsigned int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        const TopkCand v = c[x];
        if (bucket_of(v.wkey) >= b_lo) out[atomicAdd(cnt, 1u)] = v;
    }
}

cudaError_t launch_cand_collect(const TopkCand *c, unsigned int n, unsigned int b_lo,
                                TopkCand *out, unsigned int *cnt, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess || n == 0) return e;
    unsigned int blocks = (n + 255) / 256;
    k_cand_collect<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(c, n, b_lo, out, cnt);
    return cudaGetLastError();
}

// (wkey, ~ij): larger digit = earlier in the output.
__device__ __forceinline__ unsigned int order_digit(const TopkCand &c, int d) {
    unsigned long long word = d < 8 ? c.wkey : ~c.ij;
    int sh = 56 - 8 * (d & 7);
    return (unsigned int)((word >> sh) & 255ull);
}

__global__ void k_topk_digit_hist(const TopkCand *__restrict__ c, unsigned int n, int digit,
                                  unsigned int *hist) {
    __shared__ unsigned int h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    for (unsigned int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        atomicAdd(&h[order_digit(c[x], digit)], 1u);
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x)
        if (h[t]) atomicAdd(&hist[t], h[t]);
}

cudaError_t launch_topk_digit_hist(const TopkCand *c, unsigned int n, int digit,
                                   unsigned int *hist, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(hist, 0, sizeof(unsigned int) * 256, s);
    if (e != cudaSuccess || n == 0) return e;
    unsigned int blocks = (n + 255) / 256;
    k_topk_digit_hist<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(c, n, digit, hist);
    return cudaGetLastError();
}

__global__ void k_topk_digit_split(const TopkCand *__restrict__ c, unsigned int n, int digit,
                                   unsigned int pivot, TopkCand *sel, unsigned int *sel_n,
                                   TopkCand *keep, unsigned int *keep_n) {
    for (unsigned int x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x) {
        TopkCand v = c[x];
        unsigned int d = order_digit(v, digit);
        if (d > pivot) sel[atomicAdd(sel_n, 1u)] = v;
        else if (d == pivot) keep[atomicAdd(keep_n, 1u)] = v;
    }
}

cudaError_t launch_topk_digit_split(const TopkCand *c, unsigned int n, int digit,
                                    unsigned int pivot, TopkCand *sel, unsigned int *sel_n,
                                    TopkCand *keep, unsigned int *keep_n, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(keep_n, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess || n == 0) return e;
    unsigned int blocks = (n + 255) / 256;
    k_topk_digit_split<<<blocks < 1024 ? blocks : 1024, 256, 0, s>>>(c, n, digit, pivot, sel,
                                                                     sel_n, keep, keep_n);
    return cudaGetLastError();
}

// One CTA sorts up to kTopkSortMax candidates by (wkey desc, ij asc) and
// writes them out.
__global__ void __launch_bounds__(1024)
k_topk_sort_write(const TopkCand *__restrict__ c, unsigned int n, unsigned int n_write,
                  int32_t *i_out, int32_t *j_out, double *w_out, double *wl_out) {
    extern __shared__ unsigned char sm[];
    unsigned long long *kw = (unsigned long long *)sm;      // wkey
    unsigned long long *kij = kw + kTopkSortMax;            // ~ij (descending sort)
    unsigned short *src = (unsigned short *)(kij + kTopkSortMax);
    int np = 1;
    while (np < (int)n) np <<= 1;
    for (int t = threadIdx.x; t < np; t += blockDim.x) {
        if (t < (int)n) {
            kw[t] = c[t].wkey;
            kij[t] = ~c[t].ij;
        } else {
            kw[t] = 0;
            kij[t] = 0;
        }
        src[t] = (unsigned short)t;
    }
    __syncthreads();
    // bitonic sort, descending by (kw, kij)
    for (int size = 2; size <= np; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < (np >> 1); t += blockDim.x) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool desc = (lo & size) == 0;
                bool lo_less = kw[lo] < kw[hi] || (kw[lo] == kw[hi] && kij[lo] < kij[hi]);
                if (lo_less == desc) {
                    unsigned long long a = kw[lo]; kw[lo] = kw[hi]; kw[hi] = a;
                    a = kij[lo]; kij[lo] = kij[hi]; kij[hi] = a;
                    unsigned short b = src[lo]; src[lo] = src[hi]; src[hi] = b;
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < (int)n_write; t += blockDim.x) {
        const TopkCand &v = c[src[t]];
        i_out[t] = (int32_t)(v.ij >> 32);
        j_out[t] = (int32_t)(uint32_t)v.ij;
        w_out[t] = v.w;
        if (wl_out) wl_out[t] = v.wl;
    }
}

cudaError_t launch_topk_sort_write(const TopkCand *c, unsigned int n, unsigned int n_write,
                                   int32_t *i_out, int32_t *j_out, double *w_out, double *wl_out,
                                   cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    size_t smem = (size_t)kTopkSortMax * (8 + 8 + 2);
    cudaError_t e = cudaFuncSetAttribute(k_topk_sort_write,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_topk_sort_write<<<1, 1024, smem, s>>>(c, n, n_write < n ? n_write : n, i_out, j_out, w_out,
                                            wl_out);
    return cudaGetLastError();
}

// Export the live slots of partitions [p0, p1): block b handles partition
// p0 + b (grid-stride), placing entries at base[p - p0] + a block cursor.
__global__ void k_export(const Slot *__restrict__ slots, const unsigned long long *part_off,
                         const unsigned long long *part_mask, uint32_t p0, uint32_t p1,
                         const unsigned long long *base, int value_type, int32_t *i_out,
                         int32_t *j_out, double *w_out, double *wl_out) {
    __shared__ unsigned int cursor;
    for (uint32_t p = p0 + blockIdx.x; p < p1; p += gridDim.x) {
        if (threadIdx.x == 0) cursor = 0;
        __syncthreads();
        const unsigned long long off = part_off[p], cap = part_mask[p] + 1ull;
        const unsigned long long b = base[p - p0];
        for (unsigned long long x = threadIdx.x; x < cap; x += blockDim.x) {
            Slot s = slots[off + x];
            if (s.key == kEmptyKey) continue;
            unsigned int at = atomicAdd(&cursor, 1u);
            double w;
            weight_key(s, value_type, w);
            i_out[b + at] = (int32_t)(s.key >> 32);
            j_out[b + at] = (int32_t)(uint32_t)s.key;
            w_out[b + at] = w;
            if (wl_out) wl_out[b + at] = weight_lower(s, value_type, w);
        }
        __syncthreads();
    }
}

cudaError_t launch_export_range(const Slot *slots, const unsigned long long *part_off,
                                const unsigned long long *part_mask, uint32_t p0, uint32_t p1,
                                const unsigned long long *base, int value_type, int32_t *i_out,
                                int32_t *j_out, double *w_out, double *wl_out, cudaStream_t s) {
    if (p1 <= p0) return cudaSuccess;
    uint32_t n = p1 - p0;
    k_export<<<n < 4096 ? n : 4096, 256, 0, s>>>(slots, part_off, part_mask, p0, p1, base,
                                                  value_type, i_out, j_out, w_out, wl_out);
    return cudaGetLastError();
}



// ---------------------------------------------------------------------------
// Top-k certified from the hot block
// ---------------------------------------------------------------------------
//
// For {0,1} inputs an entry is bounded by the degrees of its row and column:
// C(i,j) = sum_k a_k(i) b_k(j) <= min(deg_A(i), deg_B(j)).  So every entry
// with its row outside the hot rows or its column outside the hot columns is
// at most S = max(max deg_A outside the hot rows, max deg_B outside the hot
// columns).  When the k-th heaviest entry among the hot pairs (hot row x hot
// column) is above S, no other entry can enter the top k, and the top k of
// the hot pairs is the exact answer: the full-table scan is skipped.

namespace {
constexpr int kDegreeSmem = 4096;   // hot ranks counted in shared memory first
}

// deg[v] += occurrences of v in idx[0, nnz); items of hot rank r < R count
// in shared memory first (the Zipf head would serialise on a few addresses).
__global__ void k_degrees(const int32_t *__restrict__ idx, int64_t nnz, int32_t n,
                          const uint16_t *__restrict__ rank, uint32_t R,
                          const int64_t *__restrict__ items, unsigned long long *deg) {
    __shared__ unsigned int h[kDegreeSmem];
    for (uint32_t r = threadIdx.x; r < R; r += blockDim.x) h[r] = 0u;
    __syncthreads();
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = idx[x];
        if (v < 0 || v >= n) continue;
        const uint32_t r = R ? rank[v] : 0xFFFFu;
        if (r < R) atomicAdd(&h[r], 1u);
        else atomicAdd(&deg[v], 1ull);
    }
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < R; r += blockDim.x)
        if (h[r]) atomicAdd(&deg[items[r]], (unsigned long long)h[r]);
}

cudaError_t launch_degrees(const int32_t *idx, int64_t nnz, int32_t n, const uint16_t *rank,
                           uint32_t R, const int64_t *items, unsigned long long *deg,
                           int sm_count, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    if (R > (uint32_t)kDegreeSmem) R = 0;   // (hot sets are at most 4096 items)
    const int64_t want = (nnz + 1023) / 1024;
    const int grid = (int)std::min<int64_t>(want, (int64_t)sm_count * 4);
    k_degrees<<<grid > 0 ? grid : 1, 1024, 0, s>>>(idx, nnz, n, R ? rank : nullptr, R, items, deg);
    return cudaGetLastError();
}

// out[0] = max deg[v] over the v whose hot rank is >= R (atomicMax).
__global__ void k_max_outside(const unsigned long long *__restrict__ deg, int32_t n,
                              const uint16_t *__restrict__ rank, uint32_t R,
                              unsigned long long *out) {
    unsigned long long m = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        if (rank[v] >= R && deg[v] > m) m = deg[v];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long o = __shfl_down_sync(0xffffffffu, m, d);
        m = o > m ? o : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

cudaError_t launch_max_outside(const unsigned long long *deg, int32_t n, const uint16_t *rank,
                               uint32_t R, unsigned long long *out, cudaStream_t s) {
    const int grid = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 1024);
    k_max_outside<<<grid > 0 ? grid : 1, 256, 0, s>>>(deg, n, rank, R, out);
    return cudaGetLastError();
}

// Candidates: every hot pair (items_a[r], items_b[c]) present in the exact
// tables (read-only probe from its bucket), with its count.
__global__ void k_topk_hot_candidates(const Slot *__restrict__ slots,
                                      const unsigned long long *__restrict__ part_off,
                                      const unsigned long long *__restrict__ part_mask, HashPair hp,
                                      const int64_t *__restrict__ items_a,
                                      const int64_t *__restrict__ items_b, uint32_t R,
                                      int upper_only, TopkCand *out, unsigned int *count) {
    const uint64_t total = (uint64_t)R * R;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t i = (uint32_t)items_a[x / R], j = (uint32_t)items_b[x % R];
        if (upper_only && !(i < j)) continue;
        const uint32_t p = partition_hash(hp, i, j);
        const unsigned long long mask = part_mask[p];
        if (mask == ~0ull) continue;   // outside the plan's interval
        const unsigned long long key = make_key(i, j);
        const Slot *base = slots + part_off[p];
        unsigned long long h = slot_mix(key) & mask & ~3ull;
        unsigned int c = 0;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            const Slot sl = base[h];
            if (sl.key == key) {
                c = (unsigned int)sl.val;
                break;
            }
            if (sl.key == kEmptyKey) break;
            h = (h + 1) & mask;
        }
        if (!c) continue;
        TopkCand cand;
        cand.wkey = c;
        cand.ij = key;
        cand.w = (double)c;
        cand.wl = (double)c;
        out[atomicAdd(count, 1u)] = cand;
    }
}

cudaError_t launch_topk_hot_candidates(const Slot *slots, const unsigned long long *part_off,
                                       const unsigned long long *part_mask, const HashPair &hp,
                                       const int64_t *items_a, const int64_t *items_b, uint32_t R,
                                       int upper_only, TopkCand *out, unsigned int *count,
                                       cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess || R == 0) return e;
    const uint64_t total = (uint64_t)R * R;
    const int grid = (int)std::min<uint64_t>((total + 255) / 256, 8192);
    k_topk_hot_candidates<<<grid, 256, 0, s>>>(slots, part_off, part_mask, hp, items_a, items_b, R,
                                               upper_only, out, count);
    return cudaGetLastError();
}

}  // namespace crp
