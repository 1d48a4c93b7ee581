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
}

// Add v (u32 count, or the bits of a double) to entry `key` of partition p.
__device__ __forceinline__ void table_update(const TableView &tv, uint32_t p,
                                             unsigned long long key, unsigned long long v) {
    if (tv.summary) {
        summary_update(tv, p, key, v);
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
        load_bucket_keys(s, k4);
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
__device__ __forceinline__ void smem_add_comp(unsigned long long *cell, float p, float e) {
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
