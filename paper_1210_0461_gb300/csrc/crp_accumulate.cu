// Column-row accumulation kernels.
//
//  * k_sort_by_hash: for every outer product k, the entries of b_k sorted by
//    h_b (the array H_b of Lemma 1 / Figure 1 "Hash", first step).
//  * k_accumulate: the CRoP loop of Figure 1 for a set of partition groups.
//    A work item is (tile of outer products, partition group g).  For each k
//    of the tile a warp enumerates exactly the entries of a_k b_k whose hash
//    lies in group g's interval [q, q + P/G) (Lemma 1: for each i, the j with
//    h_b(j) in the cyclic window [(q - h_a(i)) mod P, +P/G) form at most two
//    runs of H_b), spreads those terms over its 32 lanes, combines equal keys
//    of the warp with __match_any_sync, and adds them into a shared-memory
//    open-addressing table.  When the table passes its fill threshold the CTA
//    flushes it into the per-partition exact tables in HBM.
#include <cuda_runtime.h>
#include <stdint.h>

#include "crp_device.cuh"
#include "crp_internal.cuh"

namespace crp {

int accumulate_block_threads() { return kThreads; }

size_t accumulate_smem_bytes(int value_type, uint32_t S) {
    size_t v = value_type == CRP_I32 ? 4 : 8;
    return (size_t)S * (8 + v) + 64;
}

// ---------------------------------------------------------------------------
// The accumulation kernel
// ---------------------------------------------------------------------------

// S is a multiple of kThreads, so every lane runs the same number of
// iterations and the warp's updates go out together.
template <int VT, bool LOCKED>
__device__ void flush_table(unsigned long long *keys, void *vals, uint32_t S,
                            const AccumulateArgs &A, unsigned long long &flushed) {
    for (uint32_t s = threadIdx.x; s < S; s += kThreads) {
        const unsigned long long key = keys[s];
        const bool has = key != kEmptyKey;
        unsigned long long v = 0;
        uint32_t p = 0;
        if (has) {
            if (VT == CRP_I32) {
                v = ((unsigned int *)vals)[s];
                ((unsigned int *)vals)[s] = 0u;
            } else {
                unsigned long long pk = ((unsigned long long *)vals)[s];
                double d = (double)__uint_as_float((unsigned int)(pk >> 32)) +
                           (double)__uint_as_float((unsigned int)pk);
                v = (unsigned long long)__double_as_longlong(d);
                ((unsigned long long *)vals)[s] = 0ull;
            }
            keys[s] = kEmptyKey;
            const uint32_t i = (uint32_t)(key >> 32), j = (uint32_t)key;
            p = partition_hash(A.hp, i, j);
            if (A.sketch) {   // Count-Sketch of the combined entry: CS[h(e)] += v s(e)
                const bool neg = sign_negative(A.sg, i, j);
                if (VT == CRP_I32)
                    atomicAdd((unsigned long long *)A.sketch + p,
                              (unsigned long long)(neg ? -(long long)v : (long long)v));
                else {
                    const double d = __longlong_as_double((long long)v);
                    atomicAdd((double *)A.sketch + p, neg ? -d : d);
                }
            }
            ++flushed;
        }
        if (LOCKED) locked_update_warp(A.tv, has, p, key, v);
        else if (has) table_update(A.tv, p, key, v);
    }
}

// VT: value type.  DIRECT: no on-chip table; every (warp-combined) term goes
// straight to its partition table in HBM.  LOCKED: the tables are locked
// Space-Saving buckets (int mode), updated by whole warps.
template <int VT, bool DIRECT, bool LOCKED>
__global__ void __launch_bounds__(kThreads, 2)
k_accumulate(AccumulateArgs A, const uint32_t *__restrict__ b_hash) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t S = DIRECT ? 0u : A.smem_slots;
    const uint32_t smask = S - 1u;
    unsigned long long *keys = (unsigned long long *)smem_raw;
    void *vals = (void *)(keys + S);
    unsigned int *ctrl = (unsigned int *)((unsigned char *)vals + (size_t)S * (VT == CRP_I32 ? 4 : 8));
    // ctrl[0] = fill, ctrl[1] = current work item
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;

    for (uint32_t s = threadIdx.x; s < S; s += kThreads) {
        keys[s] = kEmptyKey;
        if (VT == CRP_I32) ((unsigned int *)vals)[s] = 0u;
        else ((unsigned long long *)vals)[s] = 0ull;
    }
    if (threadIdx.x == 0) ctrl[0] = 0u;
    __syncthreads();

    const uint32_t threshold = DIRECT ? 0u : (3u * S) / 4u - (uint32_t)kMaxNewPerRound;
    const uint32_t P = A.hp.ha.mask + 1u;
    const uint32_t w = P / A.groups;
    const uint32_t n_groups_here = A.group_end - A.group_begin;
    const unsigned long long total_items = (unsigned long long)A.n_tiles * n_groups_here;
    unsigned long long my_terms = 0, flushed = 0;

    // Count-Sketch, per term in the direct kernel: sketch_smem copies of the
    // estimators in shared memory after the 64-byte control block (warp w
    // adds into copy w mod sketch_smem, so few warps share an address), or
    // the plan's in HBM (the on-chip-table kernel adds each combined entry
    // at its flush)
    const bool sketch = DIRECT && A.sketch != nullptr;
    unsigned long long *cs_s = (unsigned long long *)(smem_raw + 64);
    if (sketch && A.sketch_smem) {
        for (uint32_t x = threadIdx.x; x < A.sketch_smem * P; x += kThreads) cs_s[x] = 0ull;
        __syncthreads();
        cs_s += (size_t)(warp % A.sketch_smem) * P;
    }

    if (DIRECT) {
        // each warp takes its own work items (1/kWarps of a tile of outer
        // products, of one partition group): no CTA-wide barrier, so no warp
        // waits for another
        const int64_t wt = A.tile >= (uint32_t)kWarps ? A.tile / kWarps : 1;
        const unsigned long long wtiles = (unsigned long long)((A.K + wt - 1) / wt);
        const unsigned long long warp_items = wtiles * n_groups_here;
        while (true) {
            unsigned long long item = 0;
            if (lane == 0) item = atomicAdd(&A.tv.dc->work64, 1ull);
            item = __shfl_sync(kFull, item, 0);
            if (item >= warp_items) break;
            const uint32_t g = A.group_begin + (uint32_t)(item / wtiles);
            const int64_t wtile = (int64_t)(item % wtiles);
            const uint32_t q = g * w;
            WarpEnum st;
            st.k = wtile * wt - 1;
            st.k_hi = min((int64_t)A.K, (wtile + 1) * wt);
            st.kstride = 1;
            st.has_batch = false;
            st.done = false;
            st.total = 0;
            st.pos = 0;
            while (advance(st, A, b_hash, q, w, lane)) {
                uint32_t oi, j;
                float owa, wb;
                int owner;
                const bool valid = next_term(st, A, lane, VT, oi, j, owa, wb, &owner);
                const uint32_t orank = __shfl_sync(kFull, st.my_rank, owner);
                const uint32_t owrank = __shfl_sync(kFull, st.my_wrank, owner);
                const unsigned long long key = make_key(oi, j);
                const unsigned act = __ballot_sync(kFull, valid);
                my_terms += valid ? 1 : 0;
                unsigned cnt = 1;
                bool bucket = false;   // a locked-bucket update, made by the whole warp below
                if (valid) {
                    if (VT == CRP_I32) {
                        bool lead = true;
                        if (A.use_match) {
                            unsigned peers = __match_any_sync(act, key);
                            lead = lane == __ffs(peers) - 1;
                            cnt = __popc(peers);
                        }
                        if (lead && sketch) {   // CS[h(e)] += cnt s(e)
                            const long long c = sign_negative(A.sg, oi, j) ? -(long long)cnt
                                                                            : (long long)cnt;
                            const uint32_t pp = partition_hash(A.hp, oi, j);
                            if (A.sketch_smem) atomicAdd(cs_s + pp, (unsigned long long)c);
                            else atomicAdd((unsigned long long *)A.sketch + pp,
                                           (unsigned long long)c);
                        }
                        if (lead && !dense_tiers(A, orank, owrank, oi, j, cnt)) {
                            if (LOCKED) bucket = true;
                            else table_update(A.tv, partition_hash(A.hp, oi, j), key, cnt);
                            ++flushed;
                        }
                    } else {
                        const float p = __fmul_rn(owa, wb);
                        const float e = __fmaf_rn(owa, wb, -p);
                        const double d = (double)p + (double)e;
                        const uint32_t part = partition_hash(A.hp, oi, j);
                        if (sketch) {
                            const double sd = sign_negative(A.sg, oi, j) ? -d : d;
                            if (A.sketch_smem) atomicAdd((double *)cs_s + part, sd);
                            else atomicAdd((double *)A.sketch + part, sd);
                        }
                        table_update(A.tv, part, key,
                                     (unsigned long long)__double_as_longlong(d));
                        ++flushed;
                    }
                }
                if (LOCKED)   // the warp is converged here
                    locked_update_warp(A.tv, bucket, partition_hash(A.hp, oi, j), key, cnt);
            }
        }
    }

    while (!DIRECT) {
        if (threadIdx.x == 0) ctrl[1] = atomicAdd(&A.tv.dc->work_next, 1u);
        __syncthreads();
        const unsigned long long item = ctrl[1];
        __syncthreads();
        if (item >= total_items) break;
        const uint32_t g = A.group_begin + (uint32_t)(item / A.n_tiles);
        const uint64_t tile = item % A.n_tiles;
        const uint32_t q = g * w;

        WarpEnum st;
        st.k = (int64_t)tile * A.tile + warp - kWarps;
        st.k_hi = min((int64_t)A.K, (int64_t)(tile + 1) * A.tile);
        st.kstride = kWarps;
        st.has_batch = false;
        st.done = false;
        st.total = 0;
        st.pos = 0;

        while (true) {
            for (int r = 0; r < kRoundChunks; ++r) {
                if (st.done || !advance(st, A, b_hash, q, w, lane)) break;
                uint32_t oi, j;
                float owa, wb;
                const bool valid = next_term(st, A, lane, VT, oi, j, owa, wb);
                const unsigned long long key = make_key(oi, j);
                const unsigned act = __ballot_sync(kFull, valid);
                my_terms += valid ? 1 : 0;
                bool is_new = false;
                if (VT == CRP_I32) {
                    if (valid) {
                        unsigned cnt = 1;
                        bool lead = true;
                        if (A.use_match) {
                            unsigned peers = __match_any_sync(act, key);
                            lead = lane == __ffs(peers) - 1;
                            cnt = __popc(peers);
                        }
                        if (lead) {
                            uint32_t slot;
                            is_new = smem_find(keys, smask, key, slot, &A.tv.dc->status);
                            if (slot != 0xffffffffu) atomicAdd(&((unsigned int *)vals)[slot], cnt);
                        }
                    }
                } else {
                    if (valid) {
                        const float p = __fmul_rn(owa, wb);
                        const float e = __fmaf_rn(owa, wb, -p);
                        uint32_t slot;
                        is_new = smem_find(keys, smask, key, slot, &A.tv.dc->status);
                        if (slot != 0xffffffffu)
                            smem_add_comp(&((unsigned long long *)vals)[slot], p, e,
                                          &A.tv.dc->status);
                    }
                }
                const unsigned nnew = __popc(__ballot_sync(kFull, is_new));
                if (lane == 0 && nnew) atomicAdd(&ctrl[0], nnew);
            }
            const int more = __syncthreads_or(st.done ? 0 : 1);
            if (ctrl[0] >= threshold) {
                __syncthreads();
                flush_table<VT, LOCKED>(keys, vals, S, A, flushed);
                __syncthreads();
                if (threadIdx.x == 0) ctrl[0] = 0u;
                __syncthreads();
            }
            if (!more) break;
        }
    }
    if (!DIRECT) {
        __syncthreads();
        flush_table<VT, LOCKED>(keys, vals, S, A, flushed);
    }
    if (sketch && A.sketch_smem) {   // add this CTA's estimators to the plan's
        __syncthreads();
        const unsigned long long *all = (const unsigned long long *)(smem_raw + 64);
        for (uint32_t p = threadIdx.x; p < P; p += kThreads) {
            if (VT == CRP_I32) {
                unsigned long long v = 0;
                for (uint32_t c = 0; c < A.sketch_smem; ++c) v += all[(size_t)c * P + p];
                if (v) atomicAdd((unsigned long long *)A.sketch + p, v);
            } else {
                double v = 0.0;
                for (uint32_t c = 0; c < A.sketch_smem; ++c)
                    v += __longlong_as_double((long long)all[(size_t)c * P + p]);
                if (v != 0.0) atomicAdd((double *)A.sketch + p, v);
            }
        }
    }

    // aggregate counters: warp reduce then one atomic per warp
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        my_terms += __shfl_down_sync(kFull, my_terms, d);
        flushed += __shfl_down_sync(kFull, flushed, d);
    }
    if (lane == 0) {
        if (my_terms) atomicAdd(&A.tv.dc->terms, my_terms);
        if (flushed) atomicAdd(&A.tv.dc->flushed, flushed);
    }
}

template <int VT, bool DIRECT, bool LOCKED>
static cudaError_t launch_one(const AccumulateArgs &args, const uint32_t *b_hash, int grid,
                              cudaStream_t s) {
    const size_t smem =
        DIRECT ? 64 + 8 * (size_t)args.sketch_smem * ((size_t)args.hp.ha.mask + 1)
               : accumulate_smem_bytes(VT, args.smem_slots);
    cudaError_t e = cudaFuncSetAttribute(k_accumulate<VT, DIRECT, LOCKED>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_accumulate<VT, DIRECT, LOCKED><<<grid, kThreads, smem, s>>>(args, b_hash);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const AccumulateArgs &args, const uint32_t *b_hash, int grid,
                              cudaStream_t s) {
    const bool direct = args.direct != 0;
    if (direct) {   // the direct kernel's warps take items from the 64-bit counter
        cudaError_t e = cudaMemsetAsync(&args.tv.dc->work64, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) return e;
    }
    if (args.tv.summary == 2)   // locked buckets: int mode only
        return direct ? launch_one<CRP_I32, true, true>(args, b_hash, grid, s)
                      : launch_one<CRP_I32, false, true>(args, b_hash, grid, s);
    if (args.tv.value_type == CRP_I32)
        return direct ? launch_one<CRP_I32, true, false>(args, b_hash, grid, s)
                      : launch_one<CRP_I32, false, false>(args, b_hash, grid, s);
    return direct ? launch_one<CRP_F32_COMP, true, false>(args, b_hash, grid, s)
                  : launch_one<CRP_F32_COMP, false, false>(args, b_hash, grid, s);
}

template <int VT, bool DIRECT>
static int occupancy_one(uint32_t smem_slots) {
    const size_t smem = DIRECT ? 64 : accumulate_smem_bytes(VT, smem_slots);
    int n = 0;
    if (cudaFuncSetAttribute(k_accumulate<VT, DIRECT, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_accumulate<VT, DIRECT, false>, kThreads,
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

int accumulate_max_blocks_per_sm(int value_type, uint32_t smem_slots, bool direct) {
    if (value_type == CRP_I32)
        return direct ? occupancy_one<CRP_I32, true>(smem_slots)
                      : occupancy_one<CRP_I32, false>(smem_slots);
    return direct ? occupancy_one<CRP_F32_COMP, true>(smem_slots)
                  : occupancy_one<CRP_F32_COMP, false>(smem_slots);
}

// ---------------------------------------------------------------------------
// H_b: entries of each b_k sorted by h_b (bitonic sort in shared memory)
// ---------------------------------------------------------------------------

constexpr int kSortWarpMax = 512;    // per-warp segment capacity (8 warps x 4 KB static smem)
constexpr int kSortThreads = 256;
constexpr int kSortBlockMax = 16384; // per-CTA capacity for long segments

template <int CAP>
__device__ __forceinline__ void bitonic_sort_u64(unsigned long long *v, int n_pow2, int tid,
                                                 int nthreads, bool warp_only) {
    for (int size = 2; size <= n_pow2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = tid; t < (n_pow2 >> 1); t += nthreads) {
                int lo = 2 * t - (t & (stride - 1));
                int hi = lo + stride;
                bool up = (lo & size) == 0;
                unsigned long long x = v[lo], y = v[hi];
                if ((x > y) == up) { v[lo] = y; v[hi] = x; }
            }
            if (warp_only) __syncwarp(); else __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kSortThreads)
k_sort_by_hash_warp(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                    const float *__restrict__ val, int64_t K, SideHash h,
                    int32_t *__restrict__ out_idx, float *__restrict__ out_val,
                    uint32_t *__restrict__ out_hash, DevCounters *dc, unsigned int *long_list) {
    __shared__ unsigned long long buf[kSortThreads / 32][kSortWarpMax];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *v = buf[warp];
    const int64_t stride = (int64_t)gridDim.x * (kSortThreads / 32);
    for (int64_t k = (int64_t)blockIdx.x * (kSortThreads / 32) + warp; k < K; k += stride) {
        const int64_t b0 = ptr[k];
        const int n = (int)(ptr[k + 1] - b0);
        if (n == 0) continue;
        if (n > kSortWarpMax) {
            if (lane == 0) {
                unsigned int at = atomicAdd(&dc->long_n, 1u);
                long_list[at] = (unsigned int)k;
            }
            continue;
        }
        int np = 1;
        while (np < n) np <<= 1;
        for (int t = lane; t < np; t += 32) {
            if (t < n) {
                uint32_t j = (uint32_t)idx[b0 + t];
                v[t] = ((unsigned long long)side_hash(h, j) << 32) | (uint32_t)t;
            } else {
                v[t] = ~0ull;
            }
        }
        __syncwarp();
        bitonic_sort_u64<kSortWarpMax>(v, np, lane, 32, true);
        for (int t = lane; t < n; t += 32) {
            unsigned long long x = v[t];
            uint32_t src = (uint32_t)x;
            out_idx[b0 + t] = idx[b0 + src];
            out_hash[b0 + t] = (uint32_t)(x >> 32);
            if (val) out_val[b0 + t] = val[b0 + src];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(1024)
k_sort_by_hash_block(const int64_t *__restrict__ ptr, const int32_t *__restrict__ idx,
                     const float *__restrict__ val, SideHash h, int32_t *__restrict__ out_idx,
                     float *__restrict__ out_val, uint32_t *__restrict__ out_hash,
                     DevCounters *dc, const unsigned int *long_list) {
    extern __shared__ unsigned long long lv[];
    const unsigned int nlong = dc->long_n;
    for (unsigned int q = blockIdx.x; q < nlong; q += gridDim.x) {
        const int64_t k = long_list[q];
        const int64_t b0 = ptr[k];
        const int n = (int)(ptr[k + 1] - b0);
        if (n > kSortBlockMax) {
            if (threadIdx.x == 0) atomicOr(&dc->status, kStatusBadIndex);
            continue;
        }
        int np = 1;
        while (np < n) np <<= 1;
        for (int t = threadIdx.x; t < np; t += blockDim.x) {
            if (t < n) {
                uint32_t j = (uint32_t)idx[b0 + t];
                lv[t] = ((unsigned long long)side_hash(h, j) << 32) | (uint32_t)t;
            } else {
                lv[t] = ~0ull;
            }
        }
        __syncthreads();
        bitonic_sort_u64<kSortBlockMax>(lv, np, threadIdx.x, blockDim.x, false);
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            unsigned long long x = lv[t];
            uint32_t src = (uint32_t)x;
            out_idx[b0 + t] = idx[b0 + src];
            out_hash[b0 + t] = (uint32_t)(x >> 32);
            if (val) out_val[b0 + t] = val[b0 + src];
        }
        __syncthreads();
    }
}

cudaError_t launch_sort_by_hash(const int64_t *ptr, const int32_t *idx, const float *val,
                                     int64_t K, SideHash h, int32_t *out_idx, float *out_val,
                                     uint32_t *out_hash, DevCounters *dc, unsigned int *long_list,
                                     int sm_count, cudaStream_t s) {
    if (K == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(&dc->long_n, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (K + (kSortThreads / 32) - 1) / (kSortThreads / 32);
    int grid = (int)(blocks < (int64_t)sm_count * 8 ? blocks : (int64_t)sm_count * 8);
    k_sort_by_hash_warp<<<grid, kSortThreads, 0, s>>>(ptr, idx, val, K, h, out_idx, out_val,
                                                       out_hash, dc, long_list);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    size_t smem = (size_t)kSortBlockMax * sizeof(unsigned long long);
    e = cudaFuncSetAttribute(k_sort_by_hash_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    k_sort_by_hash_block<<<sm_count, 1024, smem, s>>>(ptr, idx, val, h, out_idx, out_val, out_hash,
                                                      dc, long_list);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small helpers
// ---------------------------------------------------------------------------

__global__ void k_count_terms(const int64_t *a_ptr, const int64_t *b_ptr, int64_t K,
                              unsigned long long *out) {
    unsigned long long acc = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x)
        acc += (unsigned long long)(a_ptr[k + 1] - a_ptr[k]) * (unsigned long long)(b_ptr[k + 1] - b_ptr[k]);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}

cudaError_t launch_count_terms(const int64_t *a_ptr, const int64_t *b_ptr, int64_t K,
                               unsigned long long *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || K == 0) return e;
    int grid = (int)((K + 255) / 256 < 4096 ? (K + 255) / 256 : 4096);
    k_count_terms<<<grid, 256, 0, s>>>(a_ptr, b_ptr, K, out);
    return cudaGetLastError();
}

// Empty slots, two per 32-byte store (tables start 256-byte aligned).
__global__ void k_fill_empty(Slot *slots, uint64_t n) {
    const uint64_t pairs = n >> 1;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < pairs;
         x += (uint64_t)gridDim.x * blockDim.x) {
        asm volatile("st.global.v4.u64 [%0], {%1, %2, %1, %2};"
                     :: "l"(slots + 2 * x), "l"(kEmptyKey), "l"(0ull) : "memory");
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        slots[n - 1].key = kEmptyKey;
        slots[n - 1].val = 0ull;
    }
}

cudaError_t launch_fill_empty(Slot *slots, uint64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n / 2 + 255) / 256;
    int grid = (int)(blocks < 65536 ? (blocks > 0 ? blocks : 1) : 65536);
    k_fill_empty<<<grid, 256, 0, s>>>(slots, n);
    return cudaGetLastError();
}

// Per-partition sums (int mode: sum of counts = terms of the partition) and
// live-entry counts.
__global__ void k_partition_sums(const Slot *slots, const unsigned long long *part_off,
                                 const unsigned long long *part_mask, uint32_t P, int value_type,
                                 unsigned long long *terms_out, unsigned long long *live_out) {
    for (uint32_t p = blockIdx.x; p < P; p += gridDim.x) {
        const unsigned long long off = part_off[p], cap = part_mask[p] + 1ull;
        unsigned long long t = 0, live = 0;
        for (unsigned long long x = threadIdx.x; x < cap; x += blockDim.x) {
            Slot s = slots[off + x];
            if (s.key != kEmptyKey) {
                ++live;
                if (value_type == CRP_I32) t += (unsigned int)s.val;
            }
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            t += __shfl_down_sync(kFull, t, d);
            live += __shfl_down_sync(kFull, live, d);
        }
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&terms_out[p], t);
            atomicAdd(&live_out[p], live);
        }
    }
}

cudaError_t launch_partition_sums(const Slot *slots, const unsigned long long *part_off,
                                  const unsigned long long *part_mask, uint32_t P, int value_type,
                                  unsigned long long *terms_out, unsigned long long *live_out,
                                  cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(terms_out, 0, sizeof(unsigned long long) * P, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(live_out, 0, sizeof(unsigned long long) * P, s);
    if (e != cudaSuccess) return e;
    int grid = (int)(P < 8192 ? P : 8192);
    k_partition_sums<<<grid, 256, 0, s>>>(slots, part_off, part_mask, P, value_type, terms_out,
                                          live_out);
    return cudaGetLastError();
}

// Re-insert spilled updates (after the full partitions were grown).
__global__ void k_spill_reinsert(const SpillRec *spill, uint64_t n, HashPair hp, TableView tv) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        SpillRec r = spill[x];
        uint32_t i = (uint32_t)(r.key >> 32), j = (uint32_t)r.key;
        table_update(tv, partition_hash(hp, i, j), r.key, r.val);
    }
}

cudaError_t launch_spill_reinsert(const SpillRec *spill, uint64_t n, HashPair hp, TableView tv,
                                  cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    int grid = (int)(blocks < 16384 ? blocks : 16384);
    k_spill_reinsert<<<grid, 256, 0, s>>>(spill, n, hp, tv);
    return cudaGetLastError();
}

// Move the entries of one partition's old table into its new (larger) one.
__global__ void k_rehash(const Slot *old_slots, uint64_t old_off, uint64_t old_cap, TableView tv,
                         uint64_t new_off, uint64_t new_mask) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < old_cap;
         x += (uint64_t)gridDim.x * blockDim.x) {
        Slot s = old_slots[old_off + x];
        if (s.key == kEmptyKey) continue;
        // same probe order as table_update: linear from the 4-slot bucket
        unsigned long long h = slot_mix(s.key) & new_mask & ~3ull;
        for (unsigned long long probe = 0; probe <= new_mask; ++probe) {
            Slot *d = tv.slots + new_off + h;
            unsigned long long prev = atomicCAS(&d->key, kEmptyKey, s.key);
            if (prev == kEmptyKey) {
                d->val = s.val;
                break;
            }
            h = (h + 1) & new_mask;
        }
    }
}

cudaError_t launch_rehash_partition(const Slot *old_slots, uint64_t old_off, uint64_t old_cap,
                                    TableView tv, uint64_t new_off, uint64_t new_mask,
                                    cudaStream_t s) {
    uint64_t blocks = (old_cap + 255) / 256;
    int grid = (int)(blocks < 16384 ? blocks : 16384);
    k_rehash<<<grid, 256, 0, s>>>(old_slots, old_off, old_cap, tv, new_off, new_mask);
    return cudaGetLastError();
}

// Debug validation of a compressed input: ptr[0] == 0, ptr non-decreasing,
// ptr[K] == nnz, every index in [0, n_minor).  Sets *bad on any violation.
__global__ void k_validate_ptr(const int64_t *ptr, int64_t K, int64_t nnz, unsigned int *bad) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
         k += (int64_t)gridDim.x * blockDim.x) {
        if (ptr[k + 1] < ptr[k]) atomicOr(bad, 1u);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && (ptr[0] != 0 || ptr[K] != nnz)) atomicOr(bad, 1u);
}

__global__ void k_validate_idx(const int32_t *idx, int64_t nnz, int32_t n_minor, unsigned int *bad) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
         x += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = idx[x];
        if (v < 0 || v >= n_minor) atomicOr(bad, 2u);
    }
}

cudaError_t launch_validate_sparse(const int64_t *ptr, const int32_t *idx, int64_t K, int64_t nnz,
                                   int32_t n_minor, unsigned int *bad, cudaStream_t s) {
    int64_t b1 = (K + 255) / 256;
    k_validate_ptr<<<(int)(b1 < 4096 ? (b1 > 0 ? b1 : 1) : 4096), 256, 0, s>>>(ptr, K, nnz, bad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nnz == 0) return e;
    int64_t b2 = (nnz + 255) / 256;
    k_validate_idx<<<(int)(b2 < 4096 ? b2 : 4096), 256, 0, s>>>(idx, nnz, n_minor, bad);
    return cudaGetLastError();
}

// Add a warm stripe's counts to the partition tables and clear it.  Row
// stripe (rows = 1): entry (items[r], x); column stripe: (x, items[r]).
__global__ void k_warm_flush(unsigned int *stripe, uint32_t W, int32_t n_other,
                             const int64_t *items, int rows, HashPair hp, TableView tv,
                             unsigned long long *flushed) {
    unsigned long long n = 0;
    const uint64_t total = (uint64_t)W * (uint64_t)n_other;
    // warp-uniform trip count (blockDim is a multiple of 32): the warp's
    // updates go out together
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (uint64_t base = first; base < total; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = base + (threadIdx.x & 31u);
        const unsigned int c = x < total ? stripe[x] : 0u;
        uint32_t i = 0, j = 0;
        if (c) {
            stripe[x] = 0u;
            const uint32_t w = (uint32_t)items[x / (uint64_t)n_other];
            const uint32_t o = (uint32_t)(x % (uint64_t)n_other);
            i = rows ? w : o;
            j = rows ? o : w;
            ++n;
        }
        table_update_warp(tv, c != 0u, partition_hash(hp, i, j), make_key(i, j), c);
    }
    // one atomic per warp: a counter taken by every thread serialises on one address
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n += __shfl_down_sync(0xffffffffu, n, d);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(flushed, n);
}

cudaError_t launch_warm_flush(unsigned int *stripe, uint32_t W, int32_t n_other,
                              const int64_t *items, int rows, HashPair hp, TableView tv,
                              unsigned long long *flushed, cudaStream_t s) {
    const uint64_t n = (uint64_t)W * (uint64_t)n_other;
    if (n == 0) return cudaSuccess;
    k_warm_flush<<<(int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, s>>>(
        stripe, W, n_other, items, rows, hp, tv, flushed);
    return cudaGetLastError();
}

// Add the hot block's counts to the partition tables and clear it.
__global__ void k_hot_flush(unsigned int *hot, uint32_t R, const int64_t *items_a,
                            const int64_t *items_b, HashPair hp, TableView tv,
                            unsigned long long *flushed) {
    unsigned long long n = 0;
    const uint64_t total = (uint64_t)R * R;
    // warp-uniform trip count (blockDim is a multiple of 32)
    const uint64_t first = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    for (uint64_t base = first; base < total; base += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = base + (threadIdx.x & 31u);
        const unsigned int c = x < total ? hot[x] : 0u;
        uint32_t i = 0, j = 0;
        if (c) {
            hot[x] = 0u;
            i = (uint32_t)items_a[x / R];
            j = (uint32_t)items_b[x % R];
            ++n;
        }
        table_update_warp(tv, c != 0u, partition_hash(hp, i, j), make_key(i, j), c);
    }
    // one atomic per warp: a counter taken by every thread serialises on one address
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n += __shfl_down_sync(0xffffffffu, n, d);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(flushed, n);
}

__global__ void k_reserve_cells(const unsigned int *cells, int32_t n, unsigned int *block) {
    for (int32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < n; x += gridDim.x * blockDim.x)
        block[cells[x]] = 0u;
}

cudaError_t launch_reserve_cells(const unsigned int *cells, int32_t n, unsigned int *block,
                                 uint64_t n_cells, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(block, 0xFF, n_cells * sizeof(unsigned int), s);
    if (e != cudaSuccess || n <= 0) return e;
    k_reserve_cells<<<(n + 255) / 256, 256, 0, s>>>(cells, n, block);
    return cudaGetLastError();
}

// Add the ragged reserved block's counts to the tables (the reserved
// counters) and clear them; the row of cell x is found by binary search.
__global__ void k_reserve_flush(unsigned int *block, uint64_t n_cells, const unsigned int *res_off,
                                uint32_t rows, const int64_t *items_a, const int64_t *items_b,
                                HashPair hp, TableView tv, unsigned long long *flushed) {
    unsigned long long n = 0;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_cells;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned int c = block[x];
        if (!c || c == kCellOff) continue;
        block[x] = 0u;
        uint32_t lo = 0, hi = rows;   // last row with res_off[row] <= x
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (res_off[mid] <= x) lo = mid; else hi = mid;
        }
        const uint32_t i = (uint32_t)items_a[lo], j = (uint32_t)items_b[x - res_off[lo]];
        table_update(tv, partition_hash(hp, i, j), make_key(i, j), c);
        ++n;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) n += __shfl_down_sync(0xffffffffu, n, d);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(flushed, n);
}

cudaError_t launch_reserve_flush(unsigned int *block, uint64_t n_cells, const unsigned int *res_off,
                                 uint32_t rows, const int64_t *items_a, const int64_t *items_b,
                                 HashPair hp, TableView tv, unsigned long long *flushed,
                                 cudaStream_t s) {
    if (n_cells == 0 || rows == 0) return cudaSuccess;
    const uint64_t blocks = (n_cells + 255) / 256;
    k_reserve_flush<<<(int)(blocks < 8192 ? blocks : 8192), 256, 0, s>>>(
        block, n_cells, res_off, rows, items_a, items_b, hp, tv, flushed);
    return cudaGetLastError();
}

__global__ void k_hot_ranks(uint16_t *rank, int32_t n, const int64_t *items, uint32_t R) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        rank[x] = 0xFFFFu;
    __syncthreads();
}

__global__ void k_hot_scatter(uint16_t *rank, const int64_t *items, uint32_t R) {
    for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x)
        rank[items[r]] = (uint16_t)r;
}

cudaError_t launch_hot_flush(unsigned int *hot, uint32_t R, const int64_t *items_a,
                             const int64_t *items_b, HashPair hp, TableView tv,
                             unsigned long long *flushed, cudaStream_t s) {
    const uint64_t n = (uint64_t)R * R;
    if (n == 0) return cudaSuccess;
    k_hot_flush<<<(int)((n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192), 256, 0, s>>>(
        hot, R, items_a, items_b, hp, tv, flushed);
    return cudaGetLastError();
}

cudaError_t launch_hot_ranks(uint16_t *rank, int32_t n, const int64_t *items, uint32_t R,
                             cudaStream_t s) {
    k_hot_ranks<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, s>>>(rank, n, items, R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_hot_scatter<<<(R + 255) / 256, 256, 0, s>>>(rank, items, R);
    return cudaGetLastError();
}

}  // namespace crp
