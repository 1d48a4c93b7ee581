// Device functions shared by the enumeration kernels: the partition-table
// update (HBM), the shared-memory combining table, and the per-warp Lemma 1
// enumeration of the terms of a_k b_k that hash into one interval.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "crp_internal.cuh"

namespace crp {


constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kRoundChunks = 4;                       // chunks of 32 terms per warp per round
constexpr int kMaxNewPerRound = kWarps * kRoundChunks * 32;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Partition-table update (HBM)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void spill_update(const TableView &tv, unsigned long long key,
                                             unsigned long long v) {
    unsigned long long at = atomicAdd(&tv.dc->spill_n, 1ull);
    if (at < tv.spill_cap) {
        tv.spill[at].key = key;
        tv.spill[at].val = v;
    } else {
        atomicOr(&tv.dc->status, kStatusSpillFull);
    }
}

// Summary-mode update of partition p (Space-Saving semantics, weighted):
// a recorded key gains v; a new key, while the partition holds fewer than
// hard_cap keys, is recorded with count floor + v and overestimation floor
// (the floor bounds the weight of every key not recorded); otherwise the
// update is spilled and re-inserted after the partition is compacted.
// Reserved keys (exact counters) are looked up first.
__device__ __forceinline__ void summary_update(const TableView &tv, uint32_t p,
                                               unsigned long long key, unsigned long long v) {
    if (tv.has_reserved &&
        ((tv.res_bits_a[(uint32_t)(key >> 32) >> 5] >> ((uint32_t)(key >> 32) & 31)) & 1u) &&
        ((tv.res_bits_b[(uint32_t)key >> 5] >> ((uint32_t)key & 31)) & 1u)) {
        unsigned long long h = slot_mix(key) & tv.res_mask;
        for (unsigned long long probe = 0; probe <= tv.res_mask; ++probe) {
            const Slot *s = tv.slots + tv.res_off + h;
            const unsigned long long k = s->key;
            if (k == key) {
                atomicAdd((unsigned int *)&tv.slots[tv.res_off + h].val, (unsigned int)v);
                return;
            }
            if (k == kEmptyKey) break;
            h = (h + 1) & tv.res_mask;
        }
    }
    const unsigned long long off = tv.part_off[p];
    const unsigned long long mask = tv.part_mask[p];
    unsigned long long h = slot_mix(key) & mask;
    for (unsigned long long probe = 0; probe <= mask; ++probe) {
        Slot *s = tv.slots + off + h;
        unsigned long long k = s->key;
        if (k == kEmptyKey) {
            if (*(volatile unsigned int *)&tv.live[p] >= tv.hard_cap) break;
            k = atomicCAS(&s->key, kEmptyKey, key);
            if (k == kEmptyKey) {
                atomicAdd(&tv.live[p], 1u);
                const unsigned long long fl = tv.floor[p];
                atomicAdd(&s->val, (fl << 32) | (fl + v));
                return;
            }
        }
        if (k == key) {
            atomicAdd((unsigned int *)&s->val, (unsigned int)v);
            return;
        }
        h = (h + 1) & mask;
    }
    spill_update(tv, key, v);
}

// Locked-bucket summary update of partition p: the partition is one
// Space-Saving summary of bucket_ell counters (Preliminaries, weighted
// updates), applied under the partition's lock in the order the updates
// arrive -- the sequential algorithm on one arrival order of the
// partition's stream.  A recorded key gains v; else the first empty counter
// takes (key, v, 0); else the counter of least count (ties: smallest key)
// becomes (key, min + v, min).  Counters hold the count in the low 32 bits
// of val and the overestimation in the high 32 (the summary slot format).
// The wait for the lock is bounded (TableView::lock_wait cycles of SM clock,
// about 4 s by default); past it the update is dropped and the status
// records a timeout.

// The counters of the locked bucket at b after one weighted update (the
// caller holds the bucket's lock).
__device__ __forceinline__ void bucket_apply(Slot *b, uint32_t ell, unsigned long long key,
                                             unsigned long long v) {
    uint32_t at = ell, mn_at = 0;
    unsigned long long mn_key = ~0ull;
    unsigned int mn = 0xFFFFFFFFu;
    bool empty = false;
    for (uint32_t e = 0; e < ell; ++e) {
        const unsigned long long k = __ldcg(&b[e].key);
        if (k == key) {
            at = e;
            break;
        }
        if (k == kEmptyKey) {   // counters fill in order and are never emptied
            at = e;
            empty = true;
            break;
        }
        const unsigned int c = (unsigned int)__ldcg(&b[e].val);
        if (c < mn || (c == mn && k < mn_key)) {
            mn = c;
            mn_key = k;
            mn_at = e;
        }
    }
    if (at < ell && !empty) {
        const unsigned long long val = __ldcg(&b[at].val);
        __stcg(&b[at].val, (val & 0xFFFFFFFF00000000ull) | (unsigned int)((unsigned int)val + v));
    } else if (empty) {
        __stcg(&b[at].val, (unsigned long long)(unsigned int)v);
        __stcg(&b[at].key, key);
    } else {
        __stcg(&b[mn_at].val, ((unsigned long long)mn << 32) | (unsigned int)(mn + v));
        __stcg(&b[mn_at].key, key);
    }
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *a) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_u32(const unsigned int *a) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add_u32(unsigned int *a, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(a), "r"(v) : "memory");
}

// A ticket lock per partition (locks[2p] = next ticket, locks[2p + 1] = now
// serving): waiters are served in the order they arrive, so none starves
// however many wait for one bucket, and they poll with a plain load, sleeping
// in proportion to their place in the queue.  A waiter gives up when the wait
// passes the bound or when another waiter of the plan has already given up
// (the plan then reports the timeout); returns whether the lock is held.
__device__ __forceinline__ bool bucket_lock(const TableView &tv, uint32_t p) {
    unsigned int *next = tv.locks + 2 * (size_t)p;
    unsigned int *serving = next + 1;
    const unsigned int ticket = atomicAdd(next, 1u);
    const long long t0 = clock64();
    while (true) {
        const unsigned int now = ld_acquire_u32(serving);
        if (now == ticket) return true;
        if (ld_relaxed_u32(&tv.dc->status) & kStatusTimeout) return false;
        if (clock64() - t0 > tv.lock_wait) {
            atomicOr(&tv.dc->status, kStatusTimeout);
            return false;
        }
        const unsigned int ahead = ticket - now;
        __nanosleep(ahead < 128u ? 64u * ahead : 8192u);
    }
}

__device__ __forceinline__ void bucket_unlock(const TableView &tv, uint32_t p) {
    red_release_add_u32(tv.locks + 2 * (size_t)p + 1, 1u);
}

// One thread's update of a locked bucket (a caller whose warp has no other
// lane waiting for a lock).
__device__ __forceinline__ void locked_summary_update(const TableView &tv, uint32_t p,
                                                      unsigned long long key,
                                                      unsigned long long v) {
    if (!bucket_lock(tv, p)) return;
    bucket_apply(tv.slots + tv.part_off[p], tv.bucket_ell, key, v);
    bucket_unlock(tv, p);   // a release: the counters are written before the hand-on
}

// The keys of the 4-slot bucket at s (64 bytes, 64-byte aligned: partition
// capacities are powers of two >= 64 and tables start 256-byte aligned), in
// two 32-byte loads that do not allocate in L1 (a bucket is rarely read
// twice by one SM, and L1 keeps the partition offsets and masks instead).
__device__ __forceinline__ void load_bucket_keys(const Slot *s, unsigned long long *k4) {
    unsigned long long v0, v1;
    asm volatile("ld.global.L1::no_allocate.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(k4[0]), "=l"(v0), "=l"(k4[1]), "=l"(v1)
                 : "l"(s));
    asm volatile("ld.global.L1::no_allocate.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(k4[2]), "=l"(v0), "=l"(k4[3]), "=l"(v1)
                 : "l"(s + 2));
    (void)v0;
    (void)v1;
}

// The same with an evict-last hint: the routed apply phase works through one
// group's table region at a time, and its lines should outlast the records
// streaming past them in L2 until the group is done.
__device__ __forceinline__ void load_bucket_keys_keep(const Slot *s, unsigned long long *k4) {
    unsigned long long v0, v1;
    asm volatile("ld.global.L1::no_allocate.L2::evict_last.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(k4[0]), "=l"(v0), "=l"(k4[1]), "=l"(v1)
                 : "l"(s));
    asm volatile("ld.global.L1::no_allocate.L2::evict_last.v4.u64 {%0, %1, %2, %3}, [%4];"
                 : "=l"(k4[2]), "=l"(v0), "=l"(k4[3]), "=l"(v1)
                 : "l"(s + 2));
    (void)v0;
    (void)v1;
}

// Add v (u32 count, or the bits of a double) to entry `key` of partition p.
__device__ __forceinline__ void table_update(const TableView &tv, uint32_t p,
                                             unsigned long long key, unsigned long long v) {
    if (tv.summary) {
        if (tv.summary == 2) locked_summary_update(tv, p, key, v);
        else summary_update(tv, p, key, v);
        return;
    }
    // Plain (cacheable) loads are enough here: a partition marked full stays
    // full, and a key, once written, never changes, so a stale "not full" or a
    // stale empty key only costs a probe or a failed CAS, never a wrong count.
    if (tv.part_full[p]) {
        spill_update(tv, key, v);
        return;
    }
    const unsigned long long off = tv.part_off[p];
    const unsigned long long mask = tv.part_mask[p];
    if (mask == ~0ull) {  // a partition outside the plan's interval has no slots
        atomicOr(&tv.dc->status, kStatusNotOwned);
        return;
    }
    // Linear probing from the 4-slot bucket holding slot_mix(key): the four
    // keys of a bucket (64 bytes) are loaded together, so most updates take
    // one round trip even at high load.
    unsigned long long h = slot_mix(key) & mask & ~3ull;
    for (unsigned long long probe = 0; probe <= mask; probe += 4) {
        Slot *s = tv.slots + off + h;
        unsigned long long k4[4];
        if (tv.keep_in_l2) load_bucket_keys_keep(s, k4);
        else load_bucket_keys(s, k4);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            unsigned long long k = k4[q];
            if (k == kEmptyKey) {
                k = atomicCAS(&s[q].key, kEmptyKey, key);
                if (k == kEmptyKey) k = key;
            }
            if (k == key) {
                if (tv.value_type == CRP_I32)
                    atomicAdd((unsigned int *)&s[q].val, (unsigned int)v);
                else
                    atomicAdd((double *)&s[q].val, __longlong_as_double((long long)v));
                return;
            }
        }
        h = (h + 4) & mask;
    }
    atomicOr(&tv.part_full[p], 1u);
    atomicOr(&tv.dc->status, kStatusTableFull);
    spill_update(tv, key, v);
}

// The updates of a warp (lane with `has`) into its tables.  Every lane of
// the warp must call it together.  For locked buckets the lanes that update
// one partition form a group whose first lane takes one ticket of that
// partition's lock.  Then, round after round, every group still waiting
// checks whether its ticket is served; the groups served in a round apply
// their members' updates (members of one group one after another, in lane
// order; different groups side by side) and hand their locks on in the same
// round.  No lane holds a lock from one round to the next, so lanes of one
// warp never wait for each other, and the waits of the groups overlap.
__device__ __forceinline__ void locked_update_warp(const TableView &tv, bool has, uint32_t p,
                                                unsigned long long key, unsigned long long v) {
    if (!__ballot_sync(0xffffffffu, has)) return;
    const int lane = threadIdx.x & 31;
    const unsigned peers = __match_any_sync(0xffffffffu, has ? p : 0xFFFFFFFFu);
    const int first = __ffs(peers) - 1;
    const bool leader = has && lane == first;
    const unsigned rank = __popc(peers & ((1u << lane) - 1u));   // place in the group
    const unsigned size = has ? __popc(peers) : 0u;
    unsigned int *next = tv.locks + 2 * (size_t)(has ? p : 0u);
    unsigned int *serving = next + 1;
    unsigned int ticket = 0;
    if (leader) ticket = atomicAdd(next, 1u);
    unsigned pending = __ballot_sync(0xffffffffu, leader);   // groups, by first lane
    const long long t0 = clock64();
    while (pending) {
        unsigned int ahead = 0xFFFFFFFFu;
        bool served = false;
        if (leader && ((pending >> lane) & 1u)) {
            const unsigned int now = ld_acquire_u32(serving);
            served = now == ticket;
            ahead = ticket - now;
        }
        const unsigned srv = __ballot_sync(0xffffffffu, served);
        if (srv) {
            const bool mine = has && ((srv >> first) & 1u);   // my group is served
            const unsigned rounds = __reduce_max_sync(0xffffffffu, mine ? size : 0u);
            Slot *b = tv.slots + tv.part_off[has ? p : 0u];
            for (unsigned r = 0; r < rounds; ++r) {
                if (mine && rank == r) bucket_apply(b, tv.bucket_ell, key, v);
                __syncwarp();   // each member sees the previous member's counters
            }
            if (served) {
                // a group of one: its release orders its own counter writes; a
                // larger group's members wrote too, so fence before the hand-on
                if (size > 1) __threadfence();
                red_release_add_u32(serving, 1u);
            }
            pending &= ~srv;
            continue;
        }
        // nobody served this round: give up on the bound or when the plan has
        // already failed, else sleep in proportion to the shortest queue
        bool stop = false;
        if (lane == 0)
            stop = (ld_relaxed_u32(&tv.dc->status) & kStatusTimeout) ||
                   clock64() - t0 > tv.lock_wait;
        if (__shfl_sync(0xffffffffu, stop, 0)) {
            if (lane == 0) atomicOr(&tv.dc->status, kStatusTimeout);
            return;
        }
        const unsigned int wait = __reduce_min_sync(0xffffffffu, ahead);
        __nanosleep(wait < 128u ? 64u * wait : 8192u);
    }
}

__device__ __forceinline__ void table_update_warp(const TableView &tv, bool has, uint32_t p,
                                                  unsigned long long key,
                                                  unsigned long long v) {
    if (tv.summary == 2) locked_update_warp(tv, has, p, key, v);
    else if (has) table_update(tv, p, key, v);
}

// ---------------------------------------------------------------------------
// Shared-memory combining table
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_slot(unsigned long long key, uint32_t mask) {
    return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 40) & mask;
}

// Returns true when the key was new to the table.  The caller keeps the fill
// below 75% so a free slot always exists; the probe bound is a guard only.
__device__ __forceinline__ bool smem_find(unsigned long long *keys, uint32_t mask,
                                          unsigned long long key, uint32_t &slot,
                                          unsigned int *status) {
    uint32_t h = smem_slot(key, mask);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long k = *(volatile unsigned long long *)&keys[h];
        if (k == key) { slot = h; return false; }
        if (k == kEmptyKey) {
            unsigned long long prev = atomicCAS(&keys[h], kEmptyKey, key);
            if (prev == kEmptyKey) { slot = h; return true; }
            if (prev == key) { slot = h; return false; }
        }
        h = (h + 1) & mask;
    }
    atomicOr(status, kStatusSmemProbe);
    slot = 0xffffffffu;
    return false;
}

// fp32 TwoSum (Knuth): s + t == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &t) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Add the exact product p + e into a packed (sum, compensation) fp32 pair.
__device__ __forceinline__ void smem_add_comp(unsigned long long *cell, float p, float e,
                                              unsigned int *status) {
    unsigned long long old = *(volatile unsigned long long *)cell;
    for (int guard = 0; guard < (1 << 20); ++guard) {
        float s = __uint_as_float((unsigned int)(old >> 32));
        float c = __uint_as_float((unsigned int)old);
        float s1, t1;
        two_sum(s, p, s1, t1);
        float c1 = __fadd_rn(c, __fadd_rn(t1, e));
        unsigned long long nw = ((unsigned long long)__float_as_uint(s1) << 32) | __float_as_uint(c1);
        unsigned long long prev = atomicCAS(cell, old, nw);
        if (prev == old) return;
        old = prev;
    }
    // the guard ran out: the term is lost, so the call must not succeed
    atomicOr(status, kStatusSmemProbe);
}

// ---------------------------------------------------------------------------
// Per-warp enumeration of the terms of a_k b_k that hash into one interval
// ---------------------------------------------------------------------------

struct WarpEnum {
    int64_t k, k_hi;
    int64_t a_cur, a_end, a_beg;
    int64_t b_beg;
    int32_t b_len;
    // this lane's a entry of the current batch of 32
    uint32_t my_i;
    uint32_t my_rank;          // row of my_i in the hot block, or 0xFFFF
    uint32_t my_wrank;         // row of my_i in the warm stripe, or 0xFFFF
    float my_wa;
    int32_t lo1, n1, lo2, excl;
    int32_t total, pos;
    int32_t kstride;           // outer products between this warp's (kWarps, or 1)
    bool has_batch, done;
};

__device__ __forceinline__ int32_t lower_bound_hash(const uint32_t *hb, int32_t n, uint32_t v) {
    int32_t lo = 0, hi = n;
    while (lo < hi) {
        int32_t mid = (lo + hi) >> 1;
        if (__ldg(hb + mid) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ void load_batch(WarpEnum &st, const AccumulateArgs &A,
                                           const uint32_t *b_hash, uint32_t q, uint32_t w,
                                           int lane) {
    int64_t idx = st.a_cur + lane;
    bool va = idx < st.a_end;
    int32_t c = 0;
    st.my_i = 0;
    st.my_rank = 0xFFFFu;
    st.my_wrank = 0xFFFFu;
    st.my_wa = 1.0f;
    st.lo1 = 0; st.n1 = 0; st.lo2 = 0;
    if (va) {
        st.my_i = (uint32_t)__ldg(A.a_idx + idx);
        if (A.hot_rank_a) st.my_rank = __ldg(A.hot_rank_a + st.my_i);
        if (A.warm_rank_a) st.my_wrank = __ldg(A.warm_rank_a + st.my_i);
        if (A.a_val) st.my_wa = __ldg(A.a_val + idx);
        if (A.sym_upper) {
            st.lo1 = (int32_t)(idx - st.a_beg) + 1;
            st.n1 = st.b_len - st.lo1;
            c = st.n1 > 0 ? st.n1 : 0;
        } else if (A.groups == 1) {
            st.n1 = st.b_len;
            c = st.b_len;
        } else {
            const uint32_t P = A.hp.ha.mask + 1u;
            uint32_t x = side_hash(A.hp.ha, st.my_i);
            uint32_t s = (q - x) & (P - 1u);
            uint32_t e = s + w;
            const uint32_t *hb = b_hash + st.b_beg;
            st.lo1 = lower_bound_hash(hb, st.b_len, s);
            if (e <= P) {
                int32_t hi = (e == P) ? st.b_len : lower_bound_hash(hb, st.b_len, e);
                st.n1 = hi - st.lo1;
                c = st.n1;
            } else {
                st.n1 = st.b_len - st.lo1;
                int32_t n2 = lower_bound_hash(hb, st.b_len, e - P);
                c = st.n1 + n2;
            }
        }
    }
    int32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t y = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += y;
    }
    st.total = __shfl_sync(kFull, incl, 31);
    st.excl = incl - c;
    st.pos = 0;
    st.has_batch = true;
}

// Advance to the next batch with work.  Returns false when the tile is done.
__device__ __forceinline__ bool advance(WarpEnum &st, const AccumulateArgs &A,
                                        const uint32_t *b_hash, uint32_t q, uint32_t w,
                                        int lane) {
    while (true) {
        if (st.has_batch && st.pos < st.total) return true;
        if (st.has_batch) {
            st.a_cur += 32;
            st.has_batch = false;
            if (st.a_cur < st.a_end) {
                load_batch(st, A, b_hash, q, w, lane);
                continue;
            }
        }
        st.k += st.kstride;
        if (st.k >= st.k_hi) { st.done = true; return false; }
        int64_t a0 = __ldg(A.a_ptr + st.k), a1 = __ldg(A.a_ptr + st.k + 1);
        int64_t b0 = __ldg(A.b_ptr + st.k), b1 = __ldg(A.b_ptr + st.k + 1);
        if (a1 == a0 || b1 == b0) continue;
        st.a_cur = a0;
        st.a_beg = a0;
        st.a_end = a1;
        st.b_beg = b0;
        st.b_len = (int32_t)(b1 - b0);
        load_batch(st, A, b_hash, q, w, lane);
    }
}

// One chunk of a warp's enumeration: lane t takes flattened term pos + lane of
// the current batch.  Returns the term (valid, i, j, a value, b value).
__device__ __forceinline__ bool next_term(WarpEnum &st, const AccumulateArgs &A, int lane,
                                          int value_type, uint32_t &oi, uint32_t &j, float &owa,
                                          float &wb, int *owner = nullptr) {
    const int32_t t = st.pos + lane;
    bool valid = t < st.total;
    int o = 0;
#pragma unroll
    for (int s2 = 16; s2 > 0; s2 >>= 1) {
        int32_t e = __shfl_sync(kFull, st.excl, o + s2);
        if (e <= t) o += s2;
    }
    if (owner) *owner = o;
    oi = __shfl_sync(kFull, st.my_i, o);
    owa = __shfl_sync(kFull, st.my_wa, o);
    const int32_t olo1 = __shfl_sync(kFull, st.lo1, o);
    const int32_t on1 = __shfl_sync(kFull, st.n1, o);
    const int32_t olo2 = __shfl_sync(kFull, st.lo2, o);
    const int32_t oex = __shfl_sync(kFull, st.excl, o);
    st.pos += 32;
    j = 0;
    wb = 1.0f;
    if (valid) {
        const int32_t off = t - oex;
        const int32_t m = off < on1 ? olo1 + off : olo2 + (off - on1);
        j = (uint32_t)__ldg(A.b_idx + st.b_beg + m);
        if (value_type != CRP_I32 && A.b_val) wb = __ldg(A.b_val + st.b_beg + m);
        if (A.debug_checks && (oi >= (uint32_t)A.n_rows || j >= (uint32_t)A.n_cols)) {
            atomicOr(&A.tv.dc->status, kStatusBadIndex);
            valid = false;
        }
        if (A.mode == CRP_UPPER && !(oi < j)) valid = false;
        if (A.part_lo != 0u || A.part_hi != 0xFFFFFFFFu) {
            const uint32_t p = partition_hash(A.hp, oi, j);
            if (p < A.part_lo || p >= A.part_hi) valid = false;
        }
    }
    return valid;
}

// The dense on-chip tiers of an int term: the hot block (both items hot),
// then the warm stripes (row warm, else column warm).  Returns true when the
// term was counted there.
__device__ __forceinline__ bool dense_tiers(const AccumulateArgs &A, uint32_t orank,
                                            uint32_t owrank, uint32_t i, uint32_t j,
                                            unsigned cnt) {
    if (orank < A.hot_R) {
        const uint32_t rb = __ldg(A.hot_rank_b + j);
        if (A.resv_len) {
            // ragged reserved block: cells that are off never change, so a
            // cached read is exact
            if (rb < __ldg(A.resv_len + orank)) {
                unsigned int *c = &A.hot_block[__ldg(A.resv_off + orank) + rb];
                if (*c != kCellOff) {
                    atomicAdd(c, cnt);
                    return true;
                }
            }
        } else if (rb < A.hot_R) {
            atomicAdd(&A.hot_block[orank * A.hot_R + rb], cnt);
            return true;
        }
    }
    if (A.warm_W) {
        if (owrank < A.warm_W) {
            atomicAdd(&A.warm_a[(size_t)owrank * A.n_cols + j], cnt);
            return true;
        }
        const uint32_t wb = __ldg(A.warm_rank_b + j);
        if (wb < A.warm_W) {
            atomicAdd(&A.warm_b[(size_t)wb * A.n_rows + i], cnt);
            return true;
        }
    }
    return false;
}

}  // namespace crp
