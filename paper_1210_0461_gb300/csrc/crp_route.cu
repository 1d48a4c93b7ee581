// Two-phase exact accumulation ("routed" mode).
//
// The paper's processors each own an interval of the hash table, and the
// method runs fastest when that interval fits the processor's cache (Section
// 6, scalability on the Xeon E5570 and the Mac Pro).  On GB300 the cache that
// matters is the 126 MB L2, shared by all SMs: random atomics into an
// L2-resident region run several times faster than into HBM.  So:
//
//  1. k_route enumerates every term once (blocks of up to 32 x 32 terms of
//     a_k b_k staged in shared memory, 32 terms per warp step; for integer
//     counts of every pair each side of a block is ordered by dense-tier
//     class, so that a warp step has one destination).  Terms of hot and
//     warm items go to the dense
//     counters; every other term becomes a record appended to the bin of its
//     partition group b = h(i,j) >> shift.  (Pairs of the most frequent
//     items count first in per-CTA shared-memory counters, added into the
//     hot block at the end: their few cache lines would otherwise take the
//     bulk of the L2 atomics.)  A CTA appends to a bin through
//     its own current chunk of kChunkRecs records, taken from a shared pool:
//     one shared-memory 64-bit atomic returns (chunk, position) together, the
//     lane that receives position kChunkRecs installs the next chunk, and no
//     CTA-wide barrier is needed while enumerating.
//  2. k_apply_bulk (k_apply for real values) walks the chunks sorted by bin,
//     all warps on a few bins at a time, adding each record into its
//     partition table; a group's table region stays in L2 while it is
//     updated.
//
// An append that arrives while its chunk is being replaced backs off and
// retries; one that still finds no slot, or finds the pool exhausted, goes to
// overflow chunks that the apply phase reads like the others, and only when
// those are full straight to the tables.
#include <cuda_runtime.h>
#include <stdint.h>

#include "crp_device.cuh"
#include "crp_internal.cuh"

namespace crp {

constexpr uint32_t kNoChunk = 0xFFFFFFFFu;
// k_route runs one CTA of 1024 threads per SM: the chunks a CTA keeps open
// (one per bin) and the shared-memory core are shared by all its warps.
constexpr int kRouteThreads = 1024;
constexpr int kRouteWarps = kRouteThreads / 32;

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

// Records are read once by the apply phase: an evict-first hint keeps them
// from displacing the table region it wants in L2.  (They are written with
// plain stores: a chunk fills over time, and its lines should stay in L2
// until they are whole.)
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

// (8-byte records are stored marked evict-first in L2: many GB stream past the
// dense tiers and the open chunks' lines)
__device__ __forceinline__ void store_rec(unsigned long long *p, unsigned long long v) {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.u64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void store_rec(Rec16 *p, const Rec16 &v) {
    *(ulonglong2 *)p = *(const ulonglong2 *)&v;
}
__device__ __forceinline__ void set_empty(unsigned long long *p) { *p = kEmptyKey; }
__device__ __forceinline__ void set_empty(Rec16 *p) { p->key = kEmptyKey; }

// A chunk id from the pool, or kNoChunk when it is exhausted.  The counter is
// read first so that it grows past the pool by at most the lanes in flight.
__device__ __forceinline__ uint32_t reserve_chunk(const RouteArgs &RA) {
    if (*(volatile unsigned int *)RA.chunk_next >= RA.n_chunks) return kNoChunk;
    const uint32_t n = atomicAdd(RA.chunk_next, 1u);
    return n < RA.n_chunks ? n : kNoChunk;
}

// A record that found no chunk slot (it kept arriving while its chunk was
// being replaced, or the pool is exhausted) goes to the overflow chunks at
// the start of the pool, which the apply phase reads like any other chunk;
// once those are full, straight to its table (correct, only slower).
template <typename R>
__device__ __forceinline__ void overflow_append(const RouteArgs &RA, const R &r) {
    const unsigned int pos = atomicAdd(RA.ov_next, 1u);
    if (pos < RA.ov_cap) store_rec((R *)RA.pool + pos, r);
    else apply_record(RA, r);
}

// Append record r to bin b through this CTA's current chunk of the bin.
// cur[b] = (chunk << 32) | next position; nxt[b] = a chunk reserved ahead.
template <typename R>
__device__ __forceinline__ void bin_append(const RouteArgs &RA, unsigned long long *cur,
                                           unsigned int *nxt, uint32_t b, const R &r) {
    R *pool = (R *)RA.pool;
    // an append that lands past the end while another lane installs the next
    // chunk backs off and tries again (a bounded number of times: with few
    // bins many lanes can queue behind one installation)
    for (int attempt = 0; attempt < 4096; ++attempt) {
        const unsigned long long old = atomicAdd(&cur[b], 1ull);
        const uint32_t c = (uint32_t)(old >> 32), pos = (uint32_t)old;
        if (pos < kChunkRecs) {
            store_rec(pool + (size_t)c * kChunkRecs + pos, r);
            if (pos == kChunkRecs / 2) {            // reserve the successor ahead of need
                const uint32_t n = reserve_chunk(RA);
                if (n != kNoChunk) atomicCAS(&nxt[b], kNoChunk, n);   // a spare stays unused
            }
            return;
        }
        if (pos == kChunkRecs) {                    // this lane installs the next chunk
            uint32_t n = atomicExch(&nxt[b], kNoChunk);
            if (n == kNoChunk) n = reserve_chunk(RA);
            if (n != kNoChunk) {
                RA.chunk_bin[n] = b;
                store_rec(pool + (size_t)n * kChunkRecs, r);
                atomicExch(&cur[b], ((unsigned long long)n << 32) | 1ull);
                return;
            }
            atomicExch(&cur[b], ((unsigned long long)kNoChunk << 32) | kChunkRecs);
            break;                                  // the pool is exhausted
        }
        __nanosleep(32u << (attempt < 3 ? attempt : 3));
    }
    overflow_append(RA, r);
}

// An input index read that does not allocate in L1 (L1 keeps the rank
// arrays of the dense tiers; the index arrays stream through once) and is
// marked evict-first in L2.
__device__ __forceinline__ uint32_t ld_idx(const int32_t *p) {
    uint32_t v;
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
                 : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// Flattened enumeration of the terms of a_k b_k: a block of up to 32 entries
// of a_k (rows) and 32 of b_k (columns), with their side hashes, dense-tier
// ranks and values, is staged in the warp's shared memory, and the lanes take
// the block's mr x mc terms in order, 32 per step (term t: row t / mc, column
// t mod mc), so every lane has a term in every step but a block's last --
// where one row per lane left a lane idle for every row short of 32 (Poisson(20)
// transactions hold ~20 items).  The warp takes tiles of outer products from a
// global counter, so warps never wait on each other for work.
// Shared memory of a route CTA: per bin its open chunk (u64) and spare (u32),
// the core counters, then (flattened enumeration) 64 staged entries per warp.
__host__ __device__ __forceinline__ size_t route_stage_offset(uint32_t B, uint32_t core_H) {
    return ((size_t)B * 12 + (size_t)core_H * (core_H + 1) * 4 + 15) & ~(size_t)15;
}
struct RowData { uint32_t i, ha, ranks; float w; };   // i = ~0u: no row; ranks: hot | warm << 16
struct ColData { uint32_t j, hb, ranks; float w; };   // j = ~0u: no column
struct FlatState {
    int64_t k, a0, b0;
    int32_t left, na, nb;
    int32_t abase, bbase;   // first row / column of the block (offsets in a_k, b_k)
    int32_t mr, mc, q;      // block size; first term of the next step
    uint32_t inv_mc;        // ceil(2^16 / mc): t / mc = (t inv_mc) >> 16 for t < 1024
    bool done;
};

__device__ __forceinline__ void fl_load_rows(FlatState &st, const AccumulateArgs &A, int lane,
                                             RowData *rows) {
    __syncwarp();   // the previous block has been read by every lane
    st.mr = min(32, st.na - st.abase);
    if (lane < st.mr) {
        const int64_t x = st.a0 + st.abase + lane;
        const uint32_t i = ld_idx(A.a_idx + x);
        RowData d = {~0u, 0u, 0xFFFFFFFFu, 1.0f};
        if (i < (uint32_t)A.n_rows) {
            d.i = i;
            d.ha = side_hash(A.hp.ha, i);
            const uint32_t r = A.hot_rank_a ? __ldg(A.hot_rank_a + i) : 0xFFFFu;
            const uint32_t w = A.warm_rank_a ? __ldg(A.warm_rank_a + i) : 0xFFFFu;
            d.ranks = r | (w << 16);
            if (A.a_val) d.w = __ldg(A.a_val + x);
        } else if (A.debug_checks) {
            atomicOr(&A.tv.dc->status, kStatusBadIndex);
        }
        rows[lane] = d;
    }
    __syncwarp();
}

__device__ __forceinline__ void fl_load_cols(FlatState &st, const AccumulateArgs &A, int lane,
                                             ColData *cols) {
    __syncwarp();
    st.mc = min(32, st.nb - st.bbase);
    st.inv_mc = (65536u + (uint32_t)st.mc - 1u) / (uint32_t)st.mc;
    st.q = 0;
    if (lane < st.mc) {
        const int64_t y = st.b0 + st.bbase + lane;
        const uint32_t j = ld_idx(A.b_idx + y);
        ColData d = {~0u, 0u, 0xFFFFFFFFu, 1.0f};
        if (j < (uint32_t)A.n_cols) {
            d.j = j;
            d.hb = side_hash(A.hp.hb, j);
            const uint32_t r = A.hot_rank_b ? __ldg(A.hot_rank_b + j) : 0xFFFFu;
            const uint32_t w = A.warm_rank_b ? __ldg(A.warm_rank_b + j) : 0xFFFFu;
            d.ranks = r | (w << 16);
            if (A.b_val) d.w = __ldg(A.b_val + y);
        } else if (A.debug_checks) {
            atomicOr(&A.tv.dc->status, kStatusBadIndex);
        }
        cols[lane] = d;
    }
    __syncwarp();
}

// Make (q < mr mc) hold for a staged block; false when the warp's work is
// exhausted.  Warp-uniform.
__device__ __forceinline__ bool fl_advance(FlatState &st, const AccumulateArgs &A, int lane,
                                           RowData *rows, ColData *cols) {
    while (true) {
        if (st.q < st.mr * st.mc) return true;
        if (st.abase < st.na) {
            st.bbase += 32;
            if (st.bbase >= st.nb) {
                st.abase += 32;
                if (st.abase >= st.na) continue;
                fl_load_rows(st, A, lane, rows);
                // with T^T T above the diagonal on sorted lists, only columns
                // after the block's first row
                st.bbase = A.sym_upper ? st.abase + 1 : 0;
                if (st.bbase >= st.nb) { st.mc = 0; st.q = 0; continue; }
            }
            fl_load_cols(st, A, lane, cols);
            continue;
        }
        if (st.left > 0) {
            ++st.k;
            --st.left;
        } else {
            unsigned int item = 0;
            if (lane == 0) item = atomicAdd(&A.tv.dc->work_next, 1u);
            item = __shfl_sync(kFull, item, 0);
            if (item >= A.n_tiles) { st.done = true; return false; }
            st.k = (int64_t)item * A.tile;
            st.left = (int32_t)(min((int64_t)A.K, st.k + (int64_t)A.tile) - st.k) - 1;
        }
        st.a0 = __ldg(A.a_ptr + st.k);
        st.na = (int32_t)(__ldg(A.a_ptr + st.k + 1) - st.a0);
        st.b0 = __ldg(A.b_ptr + st.k);
        st.nb = (int32_t)(__ldg(A.b_ptr + st.k + 1) - st.b0);
        st.abase = st.na;                       // inactive until both sides are non-empty
        st.mr = st.mc = st.q = 0;
        if (st.na == 0 || st.nb == 0) continue;
        st.abase = 0;
        fl_load_rows(st, A, lane, rows);
        st.bbase = A.sym_upper ? 1 : 0;
        if (st.bbase >= st.nb) continue;
        fl_load_cols(st, A, lane, cols);
    }
}

// ---------------------------------------------------------------------------
// Class-sorted enumeration (int counts, every pair, no partition interval,
// the warm items being the first warm_W hot ranks).  A staged block of up to
// 32 entries per side is ordered by dense-tier class -- ranks below the
// smaller of (warm_W, core_H), below the larger, below hot_R, then the other
// valid entries -- so the block's terms of one destination form one or two
// rectangles:
//   core    rows [0, nH)  x cols [0, cH)
//   hot     rows [0, nH)  x cols [cH, cR)   and rows [nH, nR) x cols [0, cR)
//   warm a  rows [0, nW)  x cols [cR, cn)
//   warm b  rows [nR, m)  x cols [0, cW)
//   record  rows [nW, nR) x cols [cR, cn)   and rows [nR, m)  x cols [cW, cn)
// (nW, nH, nR: staged rows of rank below warm_W, core_H, hot_R; m: valid
// rows; c* the same for columns).  The warp walks each rectangle 32 terms at
// a time with one destination for every lane: no per-term classification
// and no divergent branches between destinations.
struct SortedCounts { int n1, n2, nR, m; };

template <typename D>
__device__ __forceinline__ SortedCounts stage_sorted(const AccumulateArgs &A, const int32_t *idx,
                                                     int64_t base, int cnt, int32_t n_items,
                                                     const uint16_t *rank_arr, const SideHash &h,
                                                     uint32_t t1, uint32_t t2, int lane, D *dst) {
    __syncwarp();   // the previous block has been read by every lane
    uint32_t v = ~0u, hv = 0u, rk = 0xFFFFu;
    int cls = 4;    // 4: no entry, or an index out of range
    if (lane < cnt) {
        const uint32_t x = ld_idx(idx + base + lane);
        if (x < (uint32_t)n_items) {
            v = x;
            hv = side_hash(h, x);
            rk = rank_arr ? __ldg(rank_arr + x) : 0xFFFFu;
            cls = (rk >= t1) + (rk >= t2) + (rk >= A.hot_R);
        } else if (A.debug_checks) {
            atomicOr(&A.tv.dc->status, kStatusBadIndex);
        }
    }
    const unsigned m0 = __ballot_sync(kFull, cls == 0), m1 = __ballot_sync(kFull, cls == 1);
    const unsigned m2 = __ballot_sync(kFull, cls == 2), m3 = __ballot_sync(kFull, cls == 3);
    SortedCounts c;
    c.n1 = __popc(m0);
    c.n2 = c.n1 + __popc(m1);
    c.nR = c.n2 + __popc(m2);
    c.m = c.nR + __popc(m3);
    const unsigned below = (1u << lane) - 1u;
    if (cls < 4) {
        const int pos = cls == 0   ? __popc(m0 & below)
                        : cls == 1 ? c.n1 + __popc(m1 & below)
                        : cls == 2 ? c.n2 + __popc(m2 & below)
                                   : c.nR + __popc(m3 & below);
        dst[pos] = D{v, hv, rk, 1.0f};   // RowData / ColData: index, side hash, rank
    }
    __syncwarp();
    return c;
}

enum { kToCore = 0, kToHot, kToWarmA, kToWarmB, kToRecord };

// +1 into a dense-tier counter, the line marked to stay in L2 (the tiers are
// tens of MB, the records that stream past them many GB)
__device__ __forceinline__ void red_keep(unsigned int *a, unsigned long long pol) {
    asm volatile("red.global.add.L2::cache_hint.u32 [%0], 1, %1;" ::"l"(a), "l"(pol) : "memory");
}

// The terms rows [r0, r1) x cols [c0, c1) of a staged block, all bound for
// destination DST.
template <int DST>
__device__ __forceinline__ void emit_rect(const RouteArgs &RA, unsigned long long *cur,
                                          unsigned int *nxt, unsigned int *core, uint32_t Hp,
                                          const RowData *rows, const ColData *cols, int r0, int r1,
                                          int c0, int c1, int lane) {
    const int nr = r1 - r0, nc = c1 - c0;
    if (nr <= 0 || nc <= 0) return;
    const AccumulateArgs &A = RA.acc;
    const int n = nr * nc;
    const uint32_t inv = (65536u + (uint32_t)nc - 1u) / (uint32_t)nc;   // t / nc for t < 1024
    unsigned long long keep = 0;
    if constexpr (DST == kToHot || DST == kToWarmA || DST == kToWarmB)
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
    for (int q = 0; q < n; q += 32) {
        const int t = q + lane;
        if (t >= n) break;
        const int rr = (int)(((uint32_t)t * inv) >> 16);
        const RowData rd = rows[r0 + rr];
        const ColData cd = cols[c0 + t - rr * nc];
        if constexpr (DST == kToCore) {
            atomicAdd(&core[rd.ranks * Hp + cd.ranks], 1u);
        } else if constexpr (DST == kToHot) {
            red_keep(&A.hot_block[rd.ranks * A.hot_R + cd.ranks], keep);
        } else if constexpr (DST == kToWarmA) {
            red_keep(&A.warm_a[(size_t)rd.ranks * A.n_cols + cd.j], keep);
        } else if constexpr (DST == kToWarmB) {
            red_keep(&A.warm_b[(size_t)cd.ranks * A.n_rows + rd.i], keep);
        } else {
            const uint32_t p = (rd.ha + cd.hb) & A.hp.ha.mask;
            bin_append(RA, cur, nxt, p >> RA.B_shift, (unsigned long long)make_key(rd.i, cd.j));
        }
    }
}

template <int VT>
__global__ void __launch_bounds__(kRouteThreads, 1) k_route(RouteArgs RA) {
    typedef typename RecT<VT>::type R;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned long long *cur = (unsigned long long *)smem_raw;
    unsigned int *nxt = (unsigned int *)(cur + RA.B);
    unsigned int *core = nxt + RA.B;            // core_H x (core_H + 1) counters (padded rows)
    const AccumulateArgs &A = RA.acc;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t H = RA.core_H, Hp = RA.core_H + 1;
    for (uint32_t b = threadIdx.x; b < RA.B; b += kRouteThreads) {
        cur[b] = ((unsigned long long)kNoChunk << 32) | kChunkRecs;   // full: first append installs
        nxt[b] = kNoChunk;
    }
    for (uint32_t x = threadIdx.x; x < H * Hp; x += kRouteThreads) core[x] = 0u;
    __syncthreads();
    const uint32_t pmask = A.hp.ha.mask;
    const bool filter = A.part_lo != 0u || A.part_hi != 0xFFFFFFFFu;
    uint32_t my_terms = 0;   // terms of this lane (fewer than 2^32 per thread)
    // this warp's staged block: 32 rows then 32 columns
    RowData *rows = (RowData *)(smem_raw + route_stage_offset(RA.B, H)) + warp * 64;
    ColData *cols = (ColData *)(rows + 32);
    // the class-sorted walk where it applies (warp-uniform: kernel arguments)
    bool sorted = false;
    unsigned long long sorted_terms = 0;   // terms of this warp on the sorted walk
    if constexpr (VT == CRP_I32) {
        sorted = A.mode == CRP_FULL && !A.sym_upper && !filter &&
                 (A.warm_W == 0 || (A.warm_in_hot && A.warm_W <= A.hot_R));
        if (sorted) {
            const uint32_t W = A.warm_W;
            const uint32_t t1 = min(W, H), t2 = max(W, H);
            const bool w_first = W <= H;
            while (true) {
                unsigned int item = 0;
                if (lane == 0) item = atomicAdd(&A.tv.dc->work_next, 1u);
                item = __shfl_sync(kFull, item, 0);
                if (item >= A.n_tiles) break;
                const int64_t k0 = (int64_t)item * A.tile;
                const int64_t k1 = min((int64_t)A.K, k0 + (int64_t)A.tile);
                for (int64_t k = k0; k < k1; ++k) {
                    const int64_t a0 = __ldg(A.a_ptr + k), b0 = __ldg(A.b_ptr + k);
                    const int32_t na = (int32_t)(__ldg(A.a_ptr + k + 1) - a0);
                    const int32_t nb = (int32_t)(__ldg(A.b_ptr + k + 1) - b0);
                    if (na <= 0 || nb <= 0) continue;
                    for (int32_t ab = 0; ab < na; ab += 32) {
                        const SortedCounts rc =
                            stage_sorted(A, A.a_idx, a0 + ab, min(32, na - ab), A.n_rows,
                                         A.hot_rank_a, A.hp.ha, t1, t2, lane, rows);
                        const int nW = w_first ? rc.n1 : rc.n2, nH = w_first ? rc.n2 : rc.n1;
                        for (int32_t bb = 0; bb < nb; bb += 32) {
                            const SortedCounts cc =
                                stage_sorted(A, A.b_idx, b0 + bb, min(32, nb - bb), A.n_cols,
                                             A.hot_rank_b, A.hp.hb, t1, t2, lane, cols);
                            const int cW = w_first ? cc.n1 : cc.n2, cH = w_first ? cc.n2 : cc.n1;
                            emit_rect<kToCore>(RA, cur, nxt, core, Hp, rows, cols, 0, nH, 0, cH,
                                               lane);
                            emit_rect<kToHot>(RA, cur, nxt, core, Hp, rows, cols, 0, nH, cH,
                                              cc.nR, lane);
                            emit_rect<kToHot>(RA, cur, nxt, core, Hp, rows, cols, nH, rc.nR, 0,
                                              cc.nR, lane);
                            emit_rect<kToWarmA>(RA, cur, nxt, core, Hp, rows, cols, 0, nW, cc.nR,
                                                cc.m, lane);
                            emit_rect<kToWarmB>(RA, cur, nxt, core, Hp, rows, cols, rc.nR, rc.m,
                                                0, cW, lane);
                            emit_rect<kToRecord>(RA, cur, nxt, core, Hp, rows, cols, nW, rc.nR,
                                                 cc.nR, cc.m, lane);
                            emit_rect<kToRecord>(RA, cur, nxt, core, Hp, rows, cols, rc.nR, rc.m,
                                                 cW, cc.m, lane);
                            sorted_terms += (unsigned long long)rc.m * (unsigned long long)cc.m;
                        }
                    }
                }
            }
        }
    }
    FlatState fs;
    fs.k = fs.a0 = fs.b0 = 0;
    fs.left = fs.na = fs.nb = fs.abase = fs.bbase = 0;
    fs.mr = fs.mc = fs.q = 0;
    fs.inv_mc = 0;
    fs.done = sorted;   // the general walk: every case the sorted one does not take
    while (!fs.done && fl_advance(fs, A, lane, rows, cols)) {
        const int32_t t = fs.q + lane;
        const int32_t nt = fs.mr * fs.mc;
        fs.q += 32;
        int32_t r = 0, c = 0;
        if (t < nt) {
            r = (int32_t)(((uint32_t)t * fs.inv_mc) >> 16);
            c = t - r * fs.mc;
        }
        const RowData rd = rows[r];
        const ColData cd = cols[c];
        const uint32_t i = rd.i, j = cd.j;
        bool valid = t < nt && i != ~0u && j != ~0u;
        if (A.mode == CRP_UPPER && !(i < j)) valid = false;
        if (A.sym_upper && fs.bbase + c <= fs.abase + r) valid = false;
        const uint32_t p = (rd.ha + cd.hb) & pmask;
        if (filter && (p < A.part_lo || p >= A.part_hi)) valid = false;
        my_terms += valid ? 1 : 0;
        if (VT == CRP_I32 && valid) {
            const uint32_t rank = rd.ranks & 0xFFFFu, wrank = rd.ranks >> 16;
            const uint32_t rb = cd.ranks & 0xFFFFu, wbk = cd.ranks >> 16;
            if (rank < A.hot_R && rb < A.hot_R) {
                if (rank < H && rb < H) atomicAdd(&core[rank * Hp + rb], 1u);
                else atomicAdd(&A.hot_block[rank * A.hot_R + rb], 1u);
                valid = false;
            } else if (wrank < A.warm_W) {
                atomicAdd(&A.warm_a[(size_t)wrank * A.n_cols + j], 1u);
                valid = false;
            } else if (wbk < A.warm_W) {
                atomicAdd(&A.warm_b[(size_t)wbk * A.n_rows + i], 1u);
                valid = false;
            }
        }
        if (valid) {
            R rec;
            if constexpr (VT == CRP_I32) {
                rec = make_key(i, j);
            } else {
                rec.key = make_key(i, j);
                rec.p = __fmul_rn(rd.w, cd.w);
                rec.e = __fmaf_rn(rd.w, cd.w, -rec.p);
            }
            bin_append(RA, cur, nxt, p >> RA.B_shift, rec);
        }
    }
    // close this CTA's chunks: mark the unused tail of each current chunk;
    // add the core counters into the hot block
    __syncthreads();
    for (uint32_t x = threadIdx.x; x < H * H; x += kRouteThreads) {
        const uint32_t ri = x / H, rj = x - ri * H;
        const unsigned int v = core[ri * Hp + rj];
        if (v) atomicAdd(&A.hot_block[ri * A.hot_R + rj], v);
    }
    R *pool = (R *)RA.pool;
    for (uint32_t b = warp; b < RA.B; b += kRouteWarps) {
        const unsigned long long w = cur[b];
        const uint32_t c = (uint32_t)(w >> 32), pos = (uint32_t)w;
        if (c == kNoChunk) continue;
        for (uint32_t x = pos + lane; x < kChunkRecs; x += 32)
            set_empty(pool + (size_t)c * kChunkRecs + x);
    }
    unsigned long long warp_terms = my_terms;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) warp_terms += __shfl_down_sync(kFull, warp_terms, d);
    warp_terms += sorted_terms;   // (the same in every lane: lane 0 adds it)
    if (lane == 0 && warp_terms) atomicAdd(&A.tv.dc->terms, warp_terms);
}

// Chunks per bin: count[b] over the installed chunks (chunk_bin != ~0u).
__global__ void k_chunk_count(const unsigned int *chunk_bin, const unsigned int *chunk_next,
                              uint32_t n_chunks, uint32_t B, unsigned int *count) {
    extern __shared__ unsigned int hist[];
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const uint32_t used = min(*chunk_next, n_chunks);
    for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < used; c += gridDim.x * blockDim.x) {
        const unsigned int b = chunk_bin[c];
        if (b != kNoChunk) atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
        if (hist[b]) atomicAdd(&count[b], hist[b]);
}

// start[b] = chunks in bins [0, b) (exclusive scan of count, B + 1 entries);
// fill[b] = start[b].  One CTA of 1024 threads.
__global__ void __launch_bounds__(1024)
k_chunk_scan(const unsigned int *count, uint32_t B, unsigned int *start, unsigned int *fill) {
    __shared__ unsigned int part[1024];
    const uint32_t per = (B + 1023) / 1024;
    const uint32_t b0 = threadIdx.x * per;
    unsigned int local = 0;
    for (uint32_t b = b0; b < b0 + per && b < B; ++b) local += count[b];
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
        start[b] = run;
        fill[b] = run;
        run += count[b];
    }
    if (threadIdx.x == 1023) start[B] = part[1023];
}

// order[] = installed chunk ids grouped by bin.
// order[] = installed chunk ids grouped by bin.  Each CTA takes spans of
// kScatterSpan chunk ids, ranks them within their bins in shared memory and
// reserves one run per bin with a single global atomic.
constexpr uint32_t kScatterSpan = 4096;
__global__ void __launch_bounds__(1024)
k_chunk_scatter(const unsigned int *chunk_bin, const unsigned int *chunk_next, uint32_t n_chunks,
                uint32_t B, unsigned int *fill, unsigned int *order) {
    extern __shared__ unsigned int sm[];
    unsigned int *hist = sm, *base = sm + B, *pk = sm + 2 * B;   // pk: bin | rank << 13
    const uint32_t used = min(*chunk_next, n_chunks);
    for (uint32_t c0 = blockIdx.x * kScatterSpan; c0 < used; c0 += gridDim.x * kScatterSpan) {
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x) hist[b] = 0u;
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < kScatterSpan; t += blockDim.x) {
            const uint32_t c = c0 + t;
            unsigned int v = ~0u;
            if (c < used) {
                const unsigned int b = chunk_bin[c];
                if (b != kNoChunk) v = b | (atomicAdd(&hist[b], 1u) << 13);
            }
            pk[t] = v;
        }
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < B; b += blockDim.x)
            if (hist[b]) base[b] = atomicAdd(&fill[b], hist[b]);
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < kScatterSpan; t += blockDim.x) {
            const unsigned int v = pk[t];
            if (v != ~0u) order[base[v & 0x1FFFu] + (v >> 13)] = c0 + t;
        }
        __syncthreads();
    }
}

// Each warp takes one chunk at a time, in bin order (so all warps work on
// one or two groups' table regions at a time), and applies its records; no
// CTA-wide barriers.
template <int VT>
__global__ void __launch_bounds__(kThreads, 2)
k_apply(RouteArgs RA) {
    typedef typename RecT<VT>::type R;
    const R *pool = (const R *)RA.pool;
    const unsigned int total = RA.start[RA.B];
    const int lane = threadIdx.x & 31;
    unsigned long long applied = 0;
    while (true) {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(&RA.acc.tv.dc->work_next, 1u);
        item = __shfl_sync(kFull, item, 0);
        if (item >= total) break;
        const R *chunk = pool + (size_t)RA.order[item] * kChunkRecs;
        if constexpr (VT == CRP_I32) {
            // lane takes kChunkRecs / 32 consecutive records, four at a time, in
            // 32-byte loads that skip L1 and leave L2 first (records are read once)
            constexpr int kPer = kChunkRecs / 32;
            const unsigned long long *src = chunk + lane * kPer;
#pragma unroll 1
            for (int h = 0; h < kPer / 4; ++h) {
                unsigned long long r[4];
                asm volatile(
                    "ld.global.L1::no_allocate.L2::evict_first.v4.u64 {%0, %1, %2, %3}, [%4];"
                    : "=l"(r[0]), "=l"(r[1]), "=l"(r[2]), "=l"(r[3])
                    : "l"(src + 4 * h));
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    if (r[x] == kEmptyKey) continue;
                    apply_record(RA, r[x]);
                    ++applied;
                }
            }
        } else {
#pragma unroll 2
            for (uint32_t x = lane; x < kChunkRecs; x += 32) {
                const R r = load_stream(chunk + x);
                if (rec_key(r) == kEmptyKey) continue;
                apply_record(RA, r);
                ++applied;
            }
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) applied += __shfl_down_sync(kFull, applied, d);
    if (lane == 0 && applied) atomicAdd(&RA.acc.tv.dc->flushed, applied);
}

// The same apply phase with each chunk's records brought into shared memory
// by the bulk-copy engine (cp.async.bulk, completion on an mbarrier).  A chunk
// is read in pieces of kStageRecs records; each warp has two piece buffers, and
// the copy of its next piece (of this chunk or of the next chunk it takes) is
// in flight while it applies the current one.  Every wait is bounded; a wait
// that gives up records a timeout and the warp stops (after waiting, again
// bounded, for its copy in flight).
constexpr bool kApplyBulk = true;
constexpr uint32_t kStageRecs = 256;
constexpr uint32_t kStageBytes = kStageRecs * 8;
constexpr uint32_t kPiecesPerChunk = kChunkRecs / kStageRecs;
constexpr int kApplyBulkPerSM = 3;   // CTAs per SM (2 x kStageBytes per warp each)
static_assert(kChunkRecs % kStageRecs == 0 && kStageBytes % 16 == 0, "piece size");

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void bulk_issue(uint32_t buf, const void *src, uint32_t mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                 "r"(kStageBytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(buf), "l"(src), "r"(kStageBytes), "r"(mbar) : "memory");
}

// Bounded wait for an mbarrier phase (~0.5 s); false when it gave up.
__device__ __forceinline__ bool bulk_wait(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(mbar), "r"(parity) : "memory");
        if (done) return true;
        __nanosleep(32);
    }
    return false;
}

__global__ void __launch_bounds__(kThreads, kApplyBulkPerSM) k_apply_bulk(RouteArgs RA) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long *buf = (unsigned long long *)smem_raw + (size_t)warp * 2 * kStageRecs;
    __shared__ __align__(8) unsigned long long mbar_store[kWarps * 2];
    // buffer b's mbarrier and shared address: base + b * step (kept in registers)
    const uint32_t mb0 = smem_addr(&mbar_store[2 * warp]), sb0 = smem_addr(buf);
    const unsigned long long *pool = (const unsigned long long *)RA.pool;
    const unsigned int total = RA.start[RA.B];
    if (lane == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    // a piece: (position in order[], piece of that chunk); item >= total: none
    auto grab = [&]() {
        unsigned int item = 0;
        if (lane == 0) item = atomicAdd(&RA.acc.tv.dc->work_next, 1u);
        return __shfl_sync(kFull, item, 0);
    };
    auto issue = [&](int b, unsigned int item, uint32_t part) {
        if (lane == 0) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            bulk_issue(sb0 + b * kStageBytes,
                       pool + (size_t)RA.order[item] * kChunkRecs + part * kStageRecs,
                       mb0 + 8 * b);
        }
    };
    unsigned long long applied = 0;
    uint32_t phases = 0u;   // bit b: the parity buffer b waits for next
    unsigned int cur_item = grab(), nxt_item = 0;
    uint32_t cur_part = 0, nxt_part = 0;
    bool pending = false;   // the next piece's copy is in flight
    if (cur_item < total) issue(0, cur_item, 0);
    if (cur_item < total) {
        nxt_item = kPiecesPerChunk > 1 ? cur_item : grab();
        nxt_part = kPiecesPerChunk > 1 ? 1u : 0u;
        if (nxt_item < total) {
            issue(1, nxt_item, nxt_part);
            pending = true;
        }
    }
    int b = 0;
    bool ok = true;
    while (cur_item < total) {
        if (!bulk_wait(mb0 + 8 * b, (phases >> b) & 1u)) { ok = false; break; }
        phases ^= 1u << b;
        const unsigned long long *rec = buf + b * kStageRecs;
#pragma unroll 1
        for (uint32_t x = lane; x < kStageRecs; x += 32) {
            const unsigned long long r = rec[x];
            if (r == kEmptyKey) continue;
            apply_record(RA, r);
            ++applied;
        }
        __syncwarp();
        // the piece after the next one goes into the buffer just freed
        cur_item = nxt_item;
        cur_part = nxt_part;
        const bool had_next = pending;
        pending = false;
        if (had_next) {
            if (cur_part + 1 < kPiecesPerChunk) {
                nxt_item = cur_item;
                nxt_part = cur_part + 1;
            } else {
                nxt_item = grab();
                nxt_part = 0;
            }
            if (nxt_item < total) {
                issue(b, nxt_item, nxt_part);
                pending = true;
            }
        } else {
            cur_item = total;   // nothing was in flight: done
        }
        b ^= 1;
    }
    if (!ok) {
        if (lane == 0) atomicOr(&RA.acc.tv.dc->status, kStatusTimeout);
        // let the copies in flight land before the warp (and its buffers) go
        bulk_wait(mb0 + 8 * b, (phases >> b) & 1u);
        if (pending) bulk_wait(mb0 + 8 * (b ^ 1), (phases >> (b ^ 1)) & 1u);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) applied += __shfl_down_sync(kFull, applied, d);
    if (lane == 0 && applied) atomicAdd(&RA.acc.tv.dc->flushed, applied);
}

size_t route_smem_bytes(uint32_t B, uint32_t core_H) {
    return route_stage_offset(B, core_H) +
           (size_t)kRouteWarps * 32 * (sizeof(RowData) + sizeof(ColData));
}

cudaError_t launch_route(const RouteArgs &RA, int grid, cudaStream_t s) {
    const size_t smem = route_smem_bytes(RA.B, RA.core_H);
    cudaError_t e;
    if (RA.acc.tv.value_type == CRP_I32) {
        e = cudaFuncSetAttribute(k_route<CRP_I32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_route<CRP_I32><<<grid, kRouteThreads, smem, s>>>(RA);
    } else {
        e = cudaFuncSetAttribute(k_route<CRP_F32_COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_route<CRP_F32_COMP><<<grid, kRouteThreads, smem, s>>>(RA);
    }
    return cudaGetLastError();
}

// Group the installed chunks by bin (count, scan, scatter), then apply them.
// count must hold B zeroed words; start B + 1, fill B.
cudaError_t launch_apply(const RouteArgs &RA, unsigned int *count, unsigned int *fill, int grid,
                         cudaStream_t s) {
    const int cgrid = grid > 0 ? grid : 1;
    k_chunk_count<<<cgrid, 1024, RA.B * sizeof(unsigned int), s>>>(
        RA.chunk_bin, RA.chunk_next, RA.n_chunks, RA.B, count);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_chunk_scan<<<1, 1024, 0, s>>>(count, RA.B, RA.start, fill);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t ssm = (2 * (size_t)RA.B + kScatterSpan) * sizeof(unsigned int);   // B <= 8192
    e = cudaFuncSetAttribute(k_chunk_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)ssm);
    if (e != cudaSuccess) return e;
    k_chunk_scatter<<<cgrid, 1024, ssm, s>>>(RA.chunk_bin, RA.chunk_next, RA.n_chunks, RA.B, fill,
                                             RA.order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&RA.acc.tv.dc->work_next, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    RouteArgs AA = RA;
    AA.acc.tv.keep_in_l2 = 1;   // the current group's table lines outlast the records
    if (RA.acc.tv.value_type == CRP_I32 && kApplyBulk) {
        const size_t sm = (size_t)kWarps * 2 * kStageBytes;
        e = cudaFuncSetAttribute(k_apply_bulk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_apply_bulk<<<grid / 2 * kApplyBulkPerSM, kThreads, sm, s>>>(AA);
    } else if (RA.acc.tv.value_type == CRP_I32)
        k_apply<CRP_I32><<<grid, kThreads, 0, s>>>(AA);
    else
        k_apply<CRP_F32_COMP><<<grid, kThreads, 0, s>>>(AA);
    return cudaGetLastError();
}

// Records of the routing phase, counted per outer product from the dense
// tiers' rank arrays: a term (i, j) is routed unless both are hot, or i or j
// is warm, so with a_k's counts L (entries), W (warm) and H (hot, not warm)
// and b_k's likewise, the records number (La - Wa)(Lb - Wb) - Ha Hb.  (An
// upper bound in CRP_UPPER mode and for interval plans.)
__device__ __forceinline__ void tier_counts(const int32_t *idx, int64_t lo, int64_t hi,
                                            const uint16_t *hot, uint32_t R, const uint16_t *warm,
                                            uint32_t W, int32_t n, long long &w, long long &h) {
    w = 0;
    h = 0;
    for (int64_t x = lo; x < hi; ++x) {
        const int32_t v = idx[x];
        if (v < 0 || v >= n) continue;
        const bool is_w = warm && warm[v] < W;
        const bool is_h = hot && hot[v] < R;
        w += is_w;
        h += is_h && !is_w;
    }
}

__global__ void k_count_records(AccumulateArgs A, unsigned long long *out) {
    unsigned long long sum = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < A.K;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a0 = A.a_ptr[k], a1 = A.a_ptr[k + 1], b0 = A.b_ptr[k], b1 = A.b_ptr[k + 1];
        long long wa = 0, ha = 0, wb = 0, hb = 0;
        if (A.hot_R || A.warm_W) {
            tier_counts(A.a_idx, a0, a1, A.hot_rank_a, A.hot_R, A.warm_rank_a, A.warm_W,
                        A.n_rows, wa, ha);
            tier_counts(A.b_idx, b0, b1, A.hot_rank_b, A.hot_R, A.warm_rank_b, A.warm_W,
                        A.n_cols, wb, hb);
        }
        const long long r = ((a1 - a0) - wa) * ((b1 - b0) - wb) - ha * hb;
        sum += (unsigned long long)(r > 0 ? r : 0);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) sum += __shfl_down_sync(kFull, sum, d);
    if ((threadIdx.x & 31) == 0 && sum) atomicAdd(out, sum);
}

cudaError_t launch_count_records(const AccumulateArgs &A, unsigned long long *out,
                                 cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    int64_t blocks = (A.K + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    if (blocks < 1) blocks = 1;
    k_count_records<<<(int)blocks, 256, 0, s>>>(A, out);
    return cudaGetLastError();
}

}  // namespace crp
