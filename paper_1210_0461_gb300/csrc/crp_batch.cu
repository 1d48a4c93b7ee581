// Many independent column-row products in one persistent, graph-captured
// launch.  Each problem q has its own CSR inputs and its own P partition
// tables; the work items (problem, tile of outer products) of all problems
// form one queue that the CTAs of a single persistent kernel drain, so
// thousands of small, uneven products keep the GPU busy without thousands of
// launches.  Tables are sized per problem from a sampling launch of the same
// kernel that keeps only the terms of partitions [0, P/Gs) (their distinct
// count, scaled by Gs, estimates the problem's entries; h is pairwise
// independent).  An optional per-problem "ready" flag lets inputs be
// published while the kernel runs; every wait on it is bounded and reports
// CRP_ETIMEOUT instead of hanging.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "crp_device.cuh"
#include "crp_internal.cuh"

namespace crp {

struct BatchProb {
    const int64_t *a_ptr;
    const int32_t *a_idx;
    const int64_t *b_ptr;
    const int32_t *b_idx;
    int64_t K;
    int32_t n_rows, n_cols;
    // dense tier (hot_R > 0): the problem's hot items per side (rank of an
    // item in its side's hot list, 0xFF when cold), their counts on the
    // sample, the lists themselves and the hot block of R x R counters; for
    // A and B the same arrays the B side shares the A side's
    uint8_t *rank_a, *rank_b;
    unsigned int *cnt_a, *cnt_b;
    int32_t *items_a, *items_b;
    unsigned int *hot;
};

struct BatchArgs {
    const BatchProb *probs;
    const unsigned long long *tile_prefix;  // [nprob + 1]
    int32_t nprob;
    uint32_t P, tile;
    int mode;
    uint32_t sample_parts;                  // > 0: keep only terms with h < sample_parts
    uint32_t hot_R;                         // > 0: pairs of two hot items count in the hot block
    const unsigned int *ready;              // nullable
    unsigned long long wait_ns;
    HashPair hp;
    TableView tv;                           // part_off/mask/full: [nprob * P]
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Each warp takes its own work items (one tile of one problem): no CTA-wide
// barrier, so no warp waits for another.
__global__ void __launch_bounds__(kThreads, 2) k_batch(BatchArgs B) {
    const int lane = threadIdx.x & 31;
    const unsigned long long total = B.tile_prefix[B.nprob];
    unsigned long long my_terms = 0, flushed = 0;
    while (true) {
        unsigned long long item = 0;
        if (lane == 0) item = atomicAdd(&B.tv.dc->work64, 1ull);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        int32_t lo = 0, hi = B.nprob;
        while (hi - lo > 1) {
            int32_t mid = (lo + hi) >> 1;
            if (B.tile_prefix[mid] <= item) lo = mid; else hi = mid;
        }
        const int32_t q = lo;
        if (B.ready) {
            int skip = 0;
            if (lane == 0 && !*(volatile const unsigned int *)&B.ready[q]) {
                const unsigned long long t0 = global_ns();
                while (!*(volatile const unsigned int *)&B.ready[q]) {
                    if (global_ns() - t0 > B.wait_ns) {
                        atomicOr(&B.tv.dc->status, kStatusTimeout);
                        skip = 1;
                        break;
                    }
                    __nanosleep(1000);
                }
            }
            if (__shfl_sync(kFull, skip, 0)) continue;
        }
        const BatchProb pr = B.probs[q];
        AccumulateArgs A;
        A.a_ptr = pr.a_ptr;
        A.a_idx = pr.a_idx;
        A.a_val = nullptr;
        A.b_ptr = pr.b_ptr;
        A.b_idx = pr.b_idx;
        A.b_val = nullptr;
        A.K = pr.K;
        A.n_rows = pr.n_rows;
        A.n_cols = pr.n_cols;
        A.groups = 1;
        A.group_begin = 0;
        A.group_end = 1;
        A.tile = B.tile;
        A.n_tiles = 0;
        A.mode = B.mode;
        A.use_match = 1;
        A.debug_checks = 0;
        A.direct = 1;
        A.smem_slots = 0;
        A.hp = B.hp;
        A.tv = B.tv;
        A.tv.part_off = B.tv.part_off + (size_t)q * B.P;
        A.tv.part_mask = B.tv.part_mask + (size_t)q * B.P;
        A.tv.part_full = B.tv.part_full + (size_t)q * B.P;
        const uint64_t tile = item - B.tile_prefix[q];
        WarpEnum st;
        st.k = (int64_t)tile * B.tile - 1;
        st.kstride = 1;
        st.k_hi = min((int64_t)pr.K, (int64_t)(tile + 1) * B.tile);
        st.has_batch = false;
        st.done = false;
        st.total = 0;
        st.pos = 0;
        while (advance(st, A, nullptr, 0u, B.P, lane)) {
            uint32_t oi, j;
            float owa, wb;
            bool valid = next_term(st, A, lane, CRP_I32, oi, j, owa, wb);
            uint32_t p = 0;
            if (valid) {
                p = partition_hash(B.hp, oi, j);
                if (B.sample_parts && p >= B.sample_parts) valid = false;
            }
            const unsigned long long key = make_key(oi, j);
            const unsigned act = __ballot_sync(kFull, valid);
            my_terms += valid ? 1 : 0;
            if (valid) {
                const unsigned peers = __match_any_sync(act, key);
                if (lane == __ffs(peers) - 1) {
                    bool dense = false;
                    if (B.hot_R) {
                        const uint32_t ra = pr.rank_a[oi], rb = pr.rank_b[j];
                        if (ra < B.hot_R && rb < B.hot_R) {
                            atomicAdd(&pr.hot[ra * B.hot_R + rb], (unsigned)__popc(peers));
                            dense = true;
                        }
                    }
                    if (!dense) {
                        table_update(A.tv, p, key, __popc(peers));
                        ++flushed;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        my_terms += __shfl_down_sync(kFull, my_terms, d);
        flushed += __shfl_down_sync(kFull, flushed, d);
    }
    if (lane == 0) {
        if (my_terms) atomicAdd(&B.tv.dc->terms, my_terms);
        if (flushed) atomicAdd(&B.tv.dc->flushed, flushed);
    }
}

// Terms per problem: sum over its outer products of |a_k| |b_k|.
__global__ void k_batch_terms(const BatchProb *probs, int32_t nprob, unsigned long long *out) {
    for (int32_t q = blockIdx.x; q < nprob; q += gridDim.x) {
        const BatchProb pr = probs[q];
        unsigned long long acc = 0;
        for (int64_t k = threadIdx.x; k < pr.K; k += blockDim.x)
            acc += (unsigned long long)(pr.a_ptr[k + 1] - pr.a_ptr[k]) *
                   (unsigned long long)(pr.b_ptr[k + 1] - pr.b_ptr[k]);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(kFull, acc, d);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&out[q], acc);
    }
}

// Dense tier of a batch, per problem (one CTA per problem): item counts over
// the first outer products (the same sample as a plan's: max(4096, K / 64)
// of them), then the hot_R most frequent items of each side (an MSD radix
// select on the counts, ties at the threshold in any order, never an item of
// count 0): their list and their rank; after the persistent kernel, the hot
// block's nonzero counters into the problem's tables.
__global__ void k_batch_item_counts(const BatchProb *probs, int32_t nprob) {
    for (int32_t q = blockIdx.x; q < nprob; q += gridDim.x) {
        const BatchProb pr = probs[q];
        if (pr.K <= 0) continue;
        const int64_t S = min(pr.K, max((int64_t)4096, pr.K / 64));
        for (int side = 0; side < 2; ++side) {
            if (side == 1 && pr.cnt_b == pr.cnt_a) break;
            const int64_t *ptr = side ? pr.b_ptr : pr.a_ptr;
            const int32_t *idx = side ? pr.b_idx : pr.a_idx;
            const int32_t n = side ? pr.n_cols : pr.n_rows;
            unsigned int *cnt = side ? pr.cnt_b : pr.cnt_a;
            const int64_t e = ptr[S];
            for (int64_t x = ptr[0] + threadIdx.x; x < e; x += blockDim.x) {
                const int32_t v = idx[x];
                if (v >= 0 && v < n) atomicAdd(&cnt[v], 1u);
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_batch_select_hot(const BatchProb *probs, int32_t nprob,
                                                          uint32_t R) {
    __shared__ unsigned int hist[256];
    __shared__ unsigned int sh_prefix, sh_need, n_taken, n_tie;
    for (int32_t q = blockIdx.x; q < nprob; q += gridDim.x) {
        const BatchProb pr = probs[q];
        for (int side = 0; side < 2; ++side) {
            if (side == 1 && pr.cnt_b == pr.cnt_a) break;
            const unsigned int *cnt = side ? pr.cnt_b : pr.cnt_a;
            const int32_t n = side ? pr.n_cols : pr.n_rows;
            int32_t *items = side ? pr.items_b : pr.items_a;
            uint8_t *rank = side ? pr.rank_b : pr.rank_a;
            uint32_t prefix = 0, pmask = 0, need = R;
            for (int pass = 0; pass < 4; ++pass) {
                const int shift = 24 - 8 * pass;
                for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[t] = 0;
                __syncthreads();
                for (int32_t x = threadIdx.x; x < n; x += blockDim.x) {
                    const uint32_t c = cnt[x];
                    if ((c & pmask) == prefix) atomicAdd(&hist[(c >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    uint32_t cum = 0;
                    int d = 255;
                    for (; d > 0; --d) {
                        if (cum + hist[d] >= need) break;
                        cum += hist[d];
                    }
                    sh_need = need - cum;
                    sh_prefix = prefix | ((uint32_t)d << shift);
                }
                __syncthreads();
                need = sh_need;
                prefix = sh_prefix;
                pmask |= 255u << shift;
                __syncthreads();
            }
            if (threadIdx.x == 0) n_taken = n_tie = 0;
            __syncthreads();
            for (int32_t x = threadIdx.x; x < n; x += blockDim.x) {
                const uint32_t c = cnt[x];
                if (c == 0) continue;
                bool take = c > prefix;
                if (c == prefix) take = atomicAdd(&n_tie, 1u) < need;
                if (take) {
                    const unsigned int pos = atomicAdd(&n_taken, 1u);   // < R by the select
                    items[pos] = x;
                    rank[x] = (uint8_t)pos;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void k_batch_hot_flush(BatchArgs B) {
    const uint32_t R = B.hot_R, RR = R * R;
    unsigned long long flushed = 0;
    for (int32_t q = blockIdx.x; q < B.nprob; q += gridDim.x) {
        const BatchProb pr = B.probs[q];
        TableView tv = B.tv;
        tv.part_off = B.tv.part_off + (size_t)q * B.P;
        tv.part_mask = B.tv.part_mask + (size_t)q * B.P;
        tv.part_full = B.tv.part_full + (size_t)q * B.P;
        for (uint32_t c = threadIdx.x; c < RR; c += blockDim.x) {
            const unsigned int v = pr.hot[c];
            if (!v) continue;
            const uint32_t i = (uint32_t)pr.items_a[c / R], j = (uint32_t)pr.items_b[c % R];
            table_update(tv, partition_hash(B.hp, i, j), make_key(i, j), v);
            ++flushed;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) flushed += __shfl_down_sync(kFull, flushed, d);
    if ((threadIdx.x & 31) == 0 && flushed) atomicAdd(&B.tv.dc->flushed, flushed);
}

// Largest live-entry count over the sampled partitions of each problem.
__global__ void k_batch_sample_live(const Slot *slots, const unsigned long long *part_off,
                                    const unsigned long long *part_mask, uint32_t P,
                                    uint32_t sample_parts, int32_t nprob,
                                    unsigned long long *max_live) {
    __shared__ unsigned long long cnt;
    for (int64_t x = blockIdx.x; x < (int64_t)nprob * sample_parts; x += gridDim.x) {
        const int32_t q = (int32_t)(x / sample_parts);
        const uint32_t p = (uint32_t)(x % sample_parts);
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        const unsigned long long off = part_off[(size_t)q * P + p];
        const unsigned long long cap = part_mask[(size_t)q * P + p] + 1ull;
        unsigned long long c = 0;
        for (unsigned long long y = threadIdx.x; y < cap; y += blockDim.x)
            c += slots[off + y].key != kEmptyKey;
        atomicAdd(&cnt, c);
        __syncthreads();
        if (threadIdx.x == 0) atomicMax(&max_live[q], cnt);
        __syncthreads();
    }
}

}  // namespace crp

using namespace crp;

struct crp_batch {
    crp_plan_desc d;
    int32_t nprob = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0, grid = 0;
    uint32_t logP = 0, tile = 64;
    HashPair hp;
    BatchProb *d_probs = nullptr;
    unsigned long long *d_tile_prefix = nullptr;
    Slot *slots = nullptr;
    uint64_t n_slots = 0;
    unsigned long long *d_off = nullptr, *d_mask = nullptr;
    unsigned int *d_full = nullptr;
    unsigned int *d_ready = nullptr;
    unsigned long long wait_ns = 0;
    DevCounters *dc = nullptr;
    SpillRec *spill = nullptr;
    std::vector<unsigned long long> h_off, h_mask, h_terms;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    uint64_t launches = 0;
    unsigned long long total_terms = 0;
    // dense tier: hot items per problem and side (R = 0: none)
    uint32_t R = 0;
    uint8_t *d_rank = nullptr;
    unsigned int *d_cnt = nullptr, *d_hot = nullptr;
    int32_t *d_items = nullptr;
    size_t rank_n = 0, items_n = 0, hot_n = 0;   // (counts: rank_n words)
};

static crp_status bfail(crp_status st, const std::string &m) {
    set_last_error(m);
    return st;
}

#define B_CUDA(call)                                                                           \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return bfail(_e == cudaErrorMemoryAllocation ? CRP_ENOMEM : CRP_ECUDA,             \
                         std::string(#call) + ": " + cudaGetErrorString(_e));                  \
    } while (0)

static uint64_t bsm64(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static uint64_t bpow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

static BatchArgs batch_args(crp_batch *b, Slot *slots, const unsigned long long *off,
                            const unsigned long long *mask, uint32_t sample_parts) {
    BatchArgs a;
    a.hot_R = sample_parts ? 0u : b->R;   // (the sizing launch counts every entry in the tables)
    a.probs = b->d_probs;
    a.tile_prefix = b->d_tile_prefix;
    a.nprob = b->nprob;
    a.P = b->d.P;
    a.tile = b->tile;
    a.mode = b->d.mode;
    a.sample_parts = sample_parts;
    a.ready = b->wait_ns ? b->d_ready : nullptr;
    a.wait_ns = b->wait_ns;
    a.hp = b->hp;
    TableView tv;
    tv.slots = slots;
    tv.part_off = off;
    tv.part_mask = mask;
    tv.part_full = b->d_full;
    tv.spill = b->spill;
    tv.spill_cap = 0;
    tv.dc = b->dc;
    tv.value_type = CRP_I32;
    a.tv = tv;
    return a;
}

static cudaError_t enqueue_run(crp_batch *b, Slot *slots, const unsigned long long *off,
                               const unsigned long long *mask, uint64_t n_slots,
                               uint32_t sample_parts) {
    cudaError_t e = launch_fill_empty(slots, n_slots, b->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->d_full, 0, (size_t)b->nprob * b->d.P * 4, b->stream);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(b->dc, 0, sizeof(DevCounters), b->stream);
    if (e != cudaSuccess) return e;
    const BatchArgs args = batch_args(b, slots, off, mask, sample_parts);
    const int pgrid = std::min(b->nprob, 65535);
    if (args.hot_R) {
        e = cudaMemsetAsync(b->d_rank, 0xFF, b->rank_n, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_cnt, 0, b->rank_n * 4, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_hot, 0, b->hot_n * 4, b->stream);
        if (e != cudaSuccess) return e;
        k_batch_item_counts<<<pgrid, 256, 0, b->stream>>>(b->d_probs, b->nprob);
        k_batch_select_hot<<<pgrid, 256, 0, b->stream>>>(b->d_probs, b->nprob, b->R);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_batch<<<b->grid, kThreads, 0, b->stream>>>(args);
    if (args.hot_R) k_batch_hot_flush<<<pgrid, 256, 0, b->stream>>>(args);
    return cudaGetLastError();
}

extern "C" void crp_batch_destroy(crp_batch *b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    cudaFree(b->d_probs);
    cudaFree(b->d_tile_prefix);
    cudaFree(b->slots);
    cudaFree(b->d_off);
    cudaFree(b->d_mask);
    cudaFree(b->d_full);
    cudaFree(b->d_ready);
    cudaFree(b->dc);
    cudaFree(b->d_rank);
    cudaFree(b->d_cnt);
    cudaFree(b->d_hot);
    cudaFree(b->d_items);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

extern "C" crp_status crp_batch_create(crp_batch **out, const crp_plan_desc *desc, int32_t nprob,
                                       const crp_sparse *A, const crp_sparse *Bm,
                                       uint64_t wait_timeout_ns, void *stream) {
    if (!out || !desc || nprob <= 0 || !A || !Bm) return bfail(CRP_EINVAL, "bad argument");
    *out = nullptr;
    const crp_plan_desc &d = *desc;
    if (!d.P || (d.P & (d.P - 1)) || d.P > 4096)
        return bfail(CRP_EINVAL, "P must be a power of two <= 4096 for batches");
    if (d.value_type != CRP_I32) return bfail(CRP_EUNSUPPORTED, "batches count {0,1} inputs");
    if (d.mode != CRP_FULL && d.mode != CRP_UPPER) return bfail(CRP_EINVAL, "unknown mode");
    std::vector<BatchProb> probs(nprob);
    std::vector<unsigned long long> tiles(nprob + 1, 0);
    crp_batch *b = new crp_batch();
    b->d = d;
    b->nprob = nprob;
    b->stream = (cudaStream_t)stream;
    b->wait_ns = wait_timeout_ns;
    b->tile = d.tile_vectors ? d.tile_vectors : 64;
    for (int32_t q = 0; q < nprob; ++q) {
        if (A[q].n_major != Bm[q].n_major || A[q].val || Bm[q].val || A[q].n_minor <= 0 ||
            Bm[q].n_minor <= 0 || (A[q].n_major > 0 && (!A[q].ptr || !Bm[q].ptr))) {
            delete b;
            return bfail(CRP_EINVAL, "problem " + std::to_string(q) + ": bad descriptor");
        }
        probs[q] = {A[q].ptr, A[q].idx, Bm[q].ptr, Bm[q].idx, A[q].n_major, A[q].n_minor,
                    Bm[q].n_minor, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        tiles[q + 1] = tiles[q] + (A[q].n_major + b->tile - 1) / b->tile;
    }
    // the dense tier (not with ready flags: it reads the inputs before the
    // persistent kernel waits for them)
    b->R = wait_timeout_ns ? 0u : std::min<uint32_t>(d.hot_items, 255u);
    std::vector<size_t> rank_at(nprob + 1, 0);
    if (b->R) {
        for (int32_t q = 0; q < nprob; ++q) {
            const bool same = A[q].ptr == Bm[q].ptr && A[q].idx == Bm[q].idx &&
                              A[q].n_minor == Bm[q].n_minor;
            rank_at[q + 1] = rank_at[q] + (size_t)A[q].n_minor + (same ? 0 : (size_t)Bm[q].n_minor);
            b->items_n += (size_t)b->R * (same ? 1 : 2);
        }
        b->rank_n = rank_at[nprob];
        b->hot_n = (size_t)nprob * b->R * b->R;
    }
    crp_status st = CRP_OK;
    auto ok = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == CRP_OK)
            st = bfail(e == cudaErrorMemoryAllocation ? CRP_ENOMEM : CRP_ECUDA,
                       std::string(what) + ": " + cudaGetErrorString(e));
        return st == CRP_OK;
    };
    int dev = 0;
    ok(cudaGetDevice(&dev), "cudaGetDevice");
    ok(cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, dev), "attr");
    int per_sm = 0;
    ok(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, kThreads, 0), "occupancy");
    b->grid = std::max(per_sm, 1) * b->sm_count;
    while ((1u << b->logP) < d.P) ++b->logP;
    uint64_t sa = d.seed_a, sb = d.seed_b;
    b->hp.ha.a = bsm64(sa);
    b->hp.ha.b = bsm64(sa);
    b->hp.hb.a = bsm64(sb);
    b->hp.hb.b = bsm64(sb);
    b->hp.ha.shift = b->hp.hb.shift = 64u - (b->logP > 0 ? b->logP : 1u);
    b->hp.ha.mask = b->hp.hb.mask = d.P - 1u;
    const size_t NP = (size_t)nprob * d.P;
    if (ok(cudaMalloc(&b->d_probs, nprob * sizeof(BatchProb)), "malloc") &&
        ok(cudaMalloc(&b->d_tile_prefix, (nprob + 1) * 8), "malloc") &&
        ok(cudaMalloc(&b->d_off, NP * 8), "malloc") && ok(cudaMalloc(&b->d_mask, NP * 8), "malloc") &&
        ok(cudaMalloc(&b->d_full, NP * 4), "malloc") && ok(cudaMalloc(&b->d_ready, nprob * 4), "malloc") &&
        ok(cudaMalloc(&b->dc, sizeof(DevCounters)), "malloc") && ok(cudaEventCreate(&b->ev0), "ev") &&
        ok(cudaEventCreate(&b->ev1), "ev")) {
        if (b->R && ok(cudaMalloc(&b->d_rank, b->rank_n), "malloc ranks") &&
            ok(cudaMalloc(&b->d_cnt, b->rank_n * 4), "malloc counts") &&
            ok(cudaMalloc(&b->d_items, b->items_n * 4), "malloc items") &&
            ok(cudaMalloc(&b->d_hot, b->hot_n * 4), "malloc hot")) {
            size_t it = 0;
            for (int32_t q = 0; q < nprob; ++q) {
                BatchProb &pr = probs[q];
                const size_t r0 = rank_at[q];
                const bool same = rank_at[q + 1] - r0 == (size_t)A[q].n_minor;
                pr.rank_a = b->d_rank + r0;
                pr.cnt_a = b->d_cnt + r0;
                pr.items_a = b->d_items + it;
                it += b->R;
                if (same) {
                    pr.rank_b = pr.rank_a;
                    pr.cnt_b = pr.cnt_a;
                    pr.items_b = pr.items_a;
                } else {
                    pr.rank_b = b->d_rank + r0 + A[q].n_minor;
                    pr.cnt_b = b->d_cnt + r0 + A[q].n_minor;
                    pr.items_b = b->d_items + it;
                    it += b->R;
                }
                pr.hot = b->d_hot + (size_t)q * b->R * b->R;
            }
        }
        ok(cudaMemcpyAsync(b->d_probs, probs.data(), nprob * sizeof(BatchProb),
                           cudaMemcpyHostToDevice, b->stream), "h2d");
        ok(cudaMemcpyAsync(b->d_tile_prefix, tiles.data(), (nprob + 1) * 8, cudaMemcpyHostToDevice,
                           b->stream), "h2d");
        ok(cudaMemsetAsync(b->d_ready, 0xff, nprob * 4, b->stream), "memset");
    }
    // terms per problem
    unsigned long long *d_terms = nullptr;
    b->h_terms.assign(nprob, 0);
    if (st == CRP_OK && ok(cudaMalloc(&d_terms, nprob * 8), "malloc")) {
        ok(cudaMemsetAsync(d_terms, 0, nprob * 8, b->stream), "memset");
        k_batch_terms<<<std::min(nprob, 65535), 256, 0, b->stream>>>(b->d_probs, nprob, d_terms);
        ok(cudaGetLastError(), "k_batch_terms");
        ok(cudaMemcpyAsync(b->h_terms.data(), d_terms, nprob * 8, cudaMemcpyDeviceToHost, b->stream),
           "d2h");
        ok(cudaStreamSynchronize(b->stream), "sync");
    }
    for (auto t : b->h_terms) b->total_terms += t;
    // sampling launch: partitions [0, P / Gs) of every problem
    const uint32_t Gs = std::min<uint32_t>(d.P, 16u);
    const uint32_t sp = d.P / Gs;
    std::vector<unsigned long long> est(nprob, 0);
    if (st == CRP_OK) {
        std::vector<unsigned long long> soff(NP, 0), smask(NP, 0);
        uint64_t total = 0;
        for (int32_t q = 0; q < nprob; ++q) {
            const uint64_t bound = std::min<uint64_t>(b->h_terms[q], (uint64_t)probs[q].n_rows *
                                                                         probs[q].n_cols);
            const uint64_t cap = bpow2(std::max<uint64_t>(2 * (bound / d.P) + 64, 64));
            for (uint32_t p = 0; p < d.P; ++p) {
                soff[(size_t)q * d.P + p] = total + (p < sp ? (uint64_t)p * cap : 0);
                smask[(size_t)q * d.P + p] = cap - 1;
            }
            total += (uint64_t)sp * cap;
        }
        Slot *tmp = nullptr;
        unsigned long long *d_ml = nullptr;
        if (ok(cudaMalloc(&tmp, total * sizeof(Slot)), "malloc sample") &&
            ok(cudaMalloc(&d_ml, nprob * 8), "malloc")) {
            ok(cudaMemcpyAsync(b->d_off, soff.data(), NP * 8, cudaMemcpyHostToDevice, b->stream), "h2d");
            ok(cudaMemcpyAsync(b->d_mask, smask.data(), NP * 8, cudaMemcpyHostToDevice, b->stream), "h2d");
            const unsigned long long saved_wait = b->wait_ns;
            b->wait_ns = 0;
            ok(enqueue_run(b, tmp, b->d_off, b->d_mask, total, sp), "sample run");
            b->wait_ns = saved_wait;
            ok(cudaMemsetAsync(d_ml, 0, nprob * 8, b->stream), "memset");
            k_batch_sample_live<<<std::min<int64_t>((int64_t)nprob * sp, 65535), 256, 0, b->stream>>>(
                tmp, b->d_off, b->d_mask, d.P, sp, nprob, d_ml);
            ok(cudaGetLastError(), "sample live");
            unsigned int status = 0;
            ok(cudaMemcpyAsync(est.data(), d_ml, nprob * 8, cudaMemcpyDeviceToHost, b->stream), "d2h");
            ok(cudaMemcpyAsync(&status, &b->dc->status, 4, cudaMemcpyDeviceToHost, b->stream), "d2h");
            ok(cudaStreamSynchronize(b->stream), "sync");
            if (st == CRP_OK && status) st = bfail(CRP_ECUDA, "sampling launch failed");
        }
        cudaFree(tmp);
        cudaFree(d_ml);
    }
    cudaFree(d_terms);
    // final tables: per problem, max sampled partition x P distinct, <= 60% load
    if (st == CRP_OK) {
        b->h_off.assign(NP, 0);
        b->h_mask.assign(NP, 0);
        uint64_t total = 0;
        for (int32_t q = 0; q < nprob; ++q) {
            const uint64_t per = (uint64_t)((double)est[q] / 0.6) + 64;
            const uint64_t cap = bpow2(per);
            for (uint32_t p = 0; p < d.P; ++p) {
                b->h_off[(size_t)q * d.P + p] = total + (uint64_t)p * cap;
                b->h_mask[(size_t)q * d.P + p] = cap - 1;
            }
            total += (uint64_t)d.P * cap;
        }
        b->n_slots = total;
        if (ok(cudaMalloc(&b->slots, total * sizeof(Slot)), "malloc tables")) {
            ok(cudaMemcpyAsync(b->d_off, b->h_off.data(), NP * 8, cudaMemcpyHostToDevice, b->stream), "h2d");
            ok(cudaMemcpyAsync(b->d_mask, b->h_mask.data(), NP * 8, cudaMemcpyHostToDevice, b->stream), "h2d");
            ok(cudaStreamSynchronize(b->stream), "sync");
        }
    }
    // capture reset + persistent kernel as one graph
    if (st == CRP_OK) {
        cudaStream_t cs = nullptr;
        cudaGraph_t g = nullptr;
        if (ok(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "stream") &&
            ok(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "capture")) {
            cudaStream_t keep = b->stream;
            b->stream = cs;
            cudaError_t e = enqueue_run(b, b->slots, b->d_off, b->d_mask, b->n_slots, 0);
            b->stream = keep;
            cudaError_t e2 = cudaStreamEndCapture(cs, &g);
            if (ok(e, "enqueue") && ok(e2, "end capture"))
                ok(cudaGraphInstantiate(&b->exec, g, 0), "instantiate");
        }
        if (g) cudaGraphDestroy(g);
        if (cs) cudaStreamDestroy(cs);
    }
    if (st != CRP_OK) {
        crp_batch_destroy(b);
        return st;
    }
    *out = b;
    return CRP_OK;
}

extern "C" crp_status crp_batch_set_ready(crp_batch *b, int32_t q, int32_t ready) {
    if (!b || q < 0 || q >= b->nprob) return bfail(CRP_EINVAL, "bad problem index");
    const unsigned int v = ready ? 1u : 0u;
    B_CUDA(cudaMemcpy(b->d_ready + q, &v, 4, cudaMemcpyHostToDevice));
    return CRP_OK;
}

extern "C" crp_status crp_batch_run(crp_batch *b) {
    if (!b) return bfail(CRP_EINVAL, "null batch");
    B_CUDA(cudaEventRecord(b->ev0, b->stream));
    B_CUDA(cudaGraphLaunch(b->exec, b->stream));
    B_CUDA(cudaEventRecord(b->ev1, b->stream));
    // table reset + persistent kernel (+ item counts, hot selection, hot flush)
    b->launches += b->R ? 5 : 2;
    return CRP_OK;
}

extern "C" crp_status crp_batch_sync(crp_batch *b, double *ms, uint64_t *terms) {
    if (!b) return bfail(CRP_EINVAL, "null batch");
    B_CUDA(cudaStreamSynchronize(b->stream));
    DevCounters dc;
    B_CUDA(cudaMemcpy(&dc, b->dc, sizeof dc, cudaMemcpyDeviceToHost));
    if (ms) {
        float f = 0.f;
        *ms = cudaEventElapsedTime(&f, b->ev0, b->ev1) == cudaSuccess ? f : 0.0;
        cudaGetLastError();
    }
    if (terms) *terms = dc.terms;
    if (dc.status & kStatusTimeout)
        return bfail(CRP_ETIMEOUT, "a problem's inputs were not marked ready in time");
    if (dc.status & (kStatusTableFull | kStatusSpillFull))
        return bfail(CRP_ETABLE_FULL, "a problem's partition table overflowed");
    if (dc.status) return bfail(CRP_ECUDA, "device status " + std::to_string(dc.status));
    return CRP_OK;
}

extern "C" crp_status crp_batch_export(crp_batch *b, int32_t q, int32_t *i_out, int32_t *j_out,
                                       double *w_out, int64_t capacity, int64_t *n_out) {
    if (!b || !n_out || q < 0 || q >= b->nprob) return bfail(CRP_EINVAL, "bad argument");
    const uint32_t P = b->d.P;
    const unsigned long long *off = b->d_off + (size_t)q * P, *mask = b->d_mask + (size_t)q * P;
    unsigned long long *d_terms = nullptr, *d_live = nullptr, *d_base = nullptr;
    B_CUDA(cudaMalloc(&d_terms, P * 8));
    B_CUDA(cudaMalloc(&d_live, P * 8));
    B_CUDA(cudaMalloc(&d_base, P * 8));
    std::vector<unsigned long long> live(P), base(P);
    B_CUDA(launch_partition_sums(b->slots, off, mask, P, CRP_I32, d_terms, d_live, b->stream));
    B_CUDA(cudaMemcpyAsync(live.data(), d_live, P * 8, cudaMemcpyDeviceToHost, b->stream));
    B_CUDA(cudaStreamSynchronize(b->stream));
    unsigned long long tot = 0;
    for (uint32_t p = 0; p < P; ++p) { base[p] = tot; tot += live[p]; }
    *n_out = (int64_t)tot;
    crp_status st = CRP_OK;
    if ((int64_t)tot > capacity) st = bfail(CRP_EINVAL, "export capacity too small");
    else if (tot) {
        int32_t *di = nullptr;
        B_CUDA(cudaMalloc(&di, tot * (4 + 4 + 8)));
        int32_t *dj = di + tot;
        double *dw = (double *)(dj + tot);
        B_CUDA(cudaMemcpyAsync(d_base, base.data(), P * 8, cudaMemcpyHostToDevice, b->stream));
        B_CUDA(launch_export_range(b->slots, off, mask, 0, P, d_base, CRP_I32, di, dj, dw, nullptr,
                                   b->stream));
        B_CUDA(cudaMemcpyAsync(i_out, di, tot * 4, cudaMemcpyDefault, b->stream));
        B_CUDA(cudaMemcpyAsync(j_out, dj, tot * 4, cudaMemcpyDefault, b->stream));
        B_CUDA(cudaMemcpyAsync(w_out, dw, tot * 8, cudaMemcpyDefault, b->stream));
        B_CUDA(cudaStreamSynchronize(b->stream));
        cudaFree(di);
    }
    cudaFree(d_terms);
    cudaFree(d_live);
    cudaFree(d_base);
    return st;
}

extern "C" crp_status crp_batch_info(const crp_batch *b, uint64_t *total_terms,
                                     uint64_t *table_slots, uint64_t *launches) {
    if (!b) return bfail(CRP_EINVAL, "null batch");
    if (total_terms) *total_terms = b->total_terms;
    if (table_slots) *table_slots = b->n_slots;
    if (launches) *launches = b->launches;
    return CRP_OK;
}
