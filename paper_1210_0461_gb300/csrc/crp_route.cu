// Two-phase exact accumulation ("routed" mode).
//
// The paper's processors each own an interval of the hash table, and the
// method runs fastest when that interval fits the processor's cache (Section
// 6, scalability on the Xeon E5570 and the Mac Pro).  On GB300 the cache that
// matters is the 126 MB L2, shared by all SMs: random atomics into an
// L2-resident region run ~8x faster than into HBM.  So:
//
//  1. k_route enumerates every term once (Lemma 1 with one interval) and
//     appends it to the bin of its partition group b = h(i,j) >> shift; the
//     appends are staged per bin in shared memory and written out in runs.
//  2. k_apply walks the bins in order, all CTAs on one bin at a time, adding
//     each record into its partition table; a group's table region (P/B
//     partitions, sized to a few tens of MB) stays in L2 while it is updated.
//
// A bin that runs out of room sends its extra records straight to the tables
// (correct, only slower).
#include <cuda_runtime.h>
#include <stdint.h>

#include "crp_device.cuh"
#include "crp_internal.cuh"

namespace crp {

constexpr int kRouteChunks = 8;   // chunks of 32 terms per warp between CTA barriers

struct Rec16 {
    unsigned long long key;
    float p, e;  // exact product p + e
};

template <int VT>
struct RecT;
template <>
struct RecT<CRP_I32> { typedef unsigned long long type; };
template <>
struct RecT<CRP_F32_COMP> { typedef Rec16 type; };

__device__ __forceinline__ unsigned long long rec_key(unsigned long long r) { return r; }
__device__ __forceinline__ unsigned long long rec_key(const Rec16 &r) { return r.key; }
__device__ __forceinline__ unsigned long long rec_val(unsigned long long) { return 1ull; }
__device__ __forceinline__ unsigned long long rec_val(const Rec16 &r) {
    return (unsigned long long)__double_as_longlong((double)r.p + (double)r.e);
}

// Records are written once and read once: evict-first hints keep them from
// displacing the table region that the apply phase wants in L2.
__device__ __forceinline__ void store_stream(unsigned long long *p, unsigned long long v) {
    __stcs(p, v);
}
__device__ __forceinline__ void store_stream(Rec16 *p, const Rec16 &v) {
    __stcs((ulonglong2 *)p, *(const ulonglong2 *)&v);
}
__device__ __forceinline__ unsigned long long load_stream(const unsigned long long *p) {
    return __ldcs(p);
}
__device__ __forceinline__ Rec16 load_stream(const Rec16 *p) {
    ulonglong2 v = __ldcs((const ulonglong2 *)p);
    return *(Rec16 *)&v;
}

template <typename R>
__device__ __forceinline__ void apply_record(const RouteArgs &RA, const R &r) {
    const unsigned long long key = rec_key(r);
    const uint32_t i = (uint32_t)(key >> 32), j = (uint32_t)key;
    table_update(RA.acc.tv, partition_hash(RA.acc.hp, i, j), key, rec_val(r));
}

template <typename R>
__device__ __forceinline__ void bin_append(const RouteArgs &RA, uint32_t b, const R &r) {
    R *bins = (R *)RA.bins;
    const unsigned long long at = atomicAdd(&RA.bin_cnt[b], 1ull);
    if (at < RA.bin_cap[b]) bins[RA.bin_off[b] + at] = r;
    else apply_record(RA, r);
}

// Write bin b's staged records out (all of them; the count is reset).
template <int VT>
__device__ __forceinline__ void flush_bin(const RouteArgs &RA, typename RecT<VT>::type *stage,
                                          unsigned int *scnt, uint32_t b, int lane) {
    typedef typename RecT<VT>::type R;
    R *bins = (R *)RA.bins;
    const uint32_t c = scnt[b];
    const uint32_t n = c < RA.R_s ? c : RA.R_s;
    if (n == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&RA.bin_cnt[b], (unsigned long long)n);
    base = __shfl_sync(kFull, base, 0);
    const unsigned long long cap = RA.bin_cap[b], off = RA.bin_off[b];
    for (uint32_t t = lane; t < n; t += 32) {
        const R r = stage[(size_t)b * RA.R_s + t];
        if (base + t < cap) store_stream(bins + off + base + t, r);
        else apply_record(RA, r);
    }
    __syncwarp();
    if (lane == 0) scnt[b] = 0;
}

template <int VT>
__global__ void __launch_bounds__(kThreads, 2) k_route(RouteArgs RA) {
    typedef typename RecT<VT>::type R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R *stage = (R *)smem_raw;
    unsigned int *scnt = (unsigned int *)(stage + (size_t)RA.B * RA.R_s);
    unsigned int *ready = scnt + RA.B;          // two lists of bins that reached the threshold
    unsigned int *ctrl = ready + 2 * RA.B;      // ctrl[0] work item, ctrl[1..2] list counts
    const AccumulateArgs &A = RA.acc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t b = threadIdx.x; b < RA.B; b += kThreads) scnt[b] = 0;
    if (threadIdx.x == 0) ctrl[1] = ctrl[2] = 0;
    __syncthreads();
    uint32_t parity = 0;
    const uint32_t thr = RA.R_s / 2 > 0 ? RA.R_s / 2 : 1;
    unsigned long long my_terms = 0;
    while (true) {
        if (threadIdx.x == 0) ctrl[0] = atomicAdd(&A.tv.dc->work_next, 1u);
        __syncthreads();
        const unsigned int item = ctrl[0];
        __syncthreads();
        if (item >= A.n_tiles) break;
        WarpEnum st;
        st.k = (int64_t)item * A.tile + warp - kWarps;
        st.k_hi = min((int64_t)A.K, (int64_t)(item + 1) * A.tile);
        st.has_batch = false;
        st.done = false;
        st.total = 0;
        st.pos = 0;
        while (true) {
            unsigned int *rlist = ready + parity * RA.B;
            unsigned int *rcount = &ctrl[1 + parity];
            for (int r = 0; r < kRouteChunks; ++r) {
                if (st.done || !advance(st, A, nullptr, 0u, A.hp.ha.mask + 1u, lane)) break;
                uint32_t oi, j;
                float owa, wb;
                int owner;
                bool valid = next_term(st, A, lane, VT, oi, j, owa, wb, &owner);
                const uint32_t orank = __shfl_sync(kFull, st.my_rank, owner);
                const uint32_t owrank = __shfl_sync(kFull, st.my_wrank, owner);
                my_terms += valid ? 1 : 0;
                if (VT == CRP_I32 && valid && dense_tiers(A, orank, owrank, oi, j, 1u))
                    valid = false;
                if (valid) {
                    const unsigned long long key = make_key(oi, j);
                    const uint32_t b = partition_hash(A.hp, oi, j) >> RA.B_shift;
                    R rec;
                    if constexpr (VT == CRP_I32) {
                        rec = key;
                    } else {
                        rec.key = key;
                        rec.p = __fmul_rn(owa, wb);
                        rec.e = __fmaf_rn(owa, wb, -rec.p);
                    }
                    const unsigned int pos = atomicAdd(&scnt[b], 1u);
                    if (pos < RA.R_s) stage[(size_t)b * RA.R_s + pos] = rec;
                    else bin_append(RA, b, rec);
                    if (pos == thr - 1) rlist[atomicAdd(rcount, 1u)] = b;
                }
            }
            const int more = __syncthreads_or(st.done ? 0 : 1);
            const unsigned int nready = *rcount;
            for (unsigned int q = warp; q < nready; q += kWarps)
                flush_bin<VT>(RA, stage, scnt, rlist[q], lane);
            if (threadIdx.x == 0) ctrl[2 - parity] = 0;   // the other list, for the next round
            parity ^= 1u;
            __syncthreads();
            if (!more) break;
        }
    }
    for (uint32_t b = warp; b < RA.B; b += kWarps) flush_bin<VT>(RA, stage, scnt, b, lane);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) my_terms += __shfl_down_sync(kFull, my_terms, d);
    if (lane == 0 && my_terms) atomicAdd(&A.tv.dc->terms, my_terms);
}

// chunk_prefix[b] = number of CH-record chunks in bins [0, b); one CTA.
__global__ void __launch_bounds__(1024)
k_bin_chunks(const unsigned long long *bin_cnt, const unsigned long long *bin_cap, uint32_t B,
             uint32_t CH, unsigned int *chunk_prefix) {
    __shared__ unsigned int part[1024];
    const uint32_t per = (B + 1023) / 1024;
    const uint32_t b0 = threadIdx.x * per;
    unsigned int local = 0;
    for (uint32_t b = b0; b < b0 + per && b < B; ++b) {
        unsigned long long n = bin_cnt[b] < bin_cap[b] ? bin_cnt[b] : bin_cap[b];
        local += (unsigned int)((n + CH - 1) / CH);
    }
    part[threadIdx.x] = local;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        unsigned int v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned int run = part[threadIdx.x] - local;
    for (uint32_t b = b0; b < b0 + per && b < B; ++b) {
        chunk_prefix[b] = run;
        unsigned long long n = bin_cnt[b] < bin_cap[b] ? bin_cnt[b] : bin_cap[b];
        run += (unsigned int)((n + CH - 1) / CH);
    }
    if (threadIdx.x == 1023) chunk_prefix[B] = part[1023];
}

// Each warp takes chunks of CH records (bins in order, so all warps work on
// one or two groups' table regions at a time) and applies them; no CTA-wide
// barriers.
template <int VT>
__global__ void __launch_bounds__(kThreads, 2)
k_apply(RouteArgs RA, const unsigned int *__restrict__ chunk_prefix, uint32_t CH) {
    typedef typename RecT<VT>::type R;
    const R *bins = (const R *)RA.bins;
    const unsigned int total = chunk_prefix[RA.B];
    const int lane = threadIdx.x & 31;
    unsigned long long applied = 0;
    while (true) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(&RA.acc.tv.dc->work_next, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        uint32_t lo = 0, hi = RA.B;
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (chunk_prefix[mid] <= item) lo = mid; else hi = mid;
        }
        const uint32_t b = lo;
        const unsigned long long n = RA.bin_cnt[b] < RA.bin_cap[b] ? RA.bin_cnt[b] : RA.bin_cap[b];
        const unsigned long long start = (unsigned long long)(item - chunk_prefix[b]) * CH;
        const unsigned long long end = start + CH < n ? start + CH : n;
        const unsigned long long off = RA.bin_off[b];
        for (unsigned long long x = start + lane; x < end; x += 32) {
            apply_record(RA, load_stream(bins + off + x));
            ++applied;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) applied += __shfl_down_sync(kFull, applied, d);
    if (lane == 0 && applied) atomicAdd(&RA.acc.tv.dc->flushed, applied);
}

size_t route_smem_bytes(int value_type, uint32_t B, uint32_t R_s) {
    const size_t rec = value_type == CRP_I32 ? 8 : 16;
    return (size_t)B * R_s * rec + (size_t)B * 12 + 16;
}

cudaError_t launch_route(const RouteArgs &RA, int grid, cudaStream_t s) {
    const size_t smem = route_smem_bytes(RA.acc.tv.value_type, RA.B, RA.R_s);
    cudaError_t e;
    if (RA.acc.tv.value_type == CRP_I32) {
        e = cudaFuncSetAttribute(k_route<CRP_I32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_route<CRP_I32><<<grid, kThreads, smem, s>>>(RA);
    } else {
        e = cudaFuncSetAttribute(k_route<CRP_F32_COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_route<CRP_F32_COMP><<<grid, kThreads, smem, s>>>(RA);
    }
    return cudaGetLastError();
}

cudaError_t launch_apply(const RouteArgs &RA, unsigned int *chunk_prefix, uint32_t CH, int grid,
                         cudaStream_t s) {
    k_bin_chunks<<<1, 1024, 0, s>>>(RA.bin_cnt, RA.bin_cap, RA.B, CH, chunk_prefix);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&RA.acc.tv.dc->work_next, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (RA.acc.tv.value_type == CRP_I32)
        k_apply<CRP_I32><<<grid, kThreads, 0, s>>>(RA, chunk_prefix, CH);
    else
        k_apply<CRP_F32_COMP><<<grid, kThreads, 0, s>>>(RA, chunk_prefix, CH);
    return cudaGetLastError();
}

}  // namespace crp
