// Internal definitions shared by the CUDA translation units of libcrp.
//
// Partition hash (Section 4, Lemma 1 proof):  h(i,j) = (h_a(i) + h_b(j)) mod P
// with multiply-add-shift side hashes h(x) = ((a x + b) mod 2^64) >> (64 - lg P),
// (a, b) the first two SplitMix64 outputs of the side's seed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/crp.h"

namespace crp {

constexpr uint64_t kEmptyKey = ~0ull;   // i, j < 2^31 so no real key is all ones
constexpr unsigned int kCellOff = 0xFFFFFFFFu;   // a dense-block cell that is not counted
constexpr uint32_t kStatusTableFull = 1u;
constexpr uint32_t kStatusSpillFull = 2u;
constexpr uint32_t kStatusBadIndex = 4u;
constexpr uint32_t kStatusTimeout = 8u;
constexpr uint32_t kStatusSmemProbe = 16u;
constexpr uint32_t kStatusNotOwned = 32u;
// Value-type code of summary slots inside the top-k / export kernels:
// low 32 bits = count (upper bound), high 32 bits = overestimation.
constexpr int kVTSummary = 2;

// One side hash, branch-free for P = 1: (v >> (64 - max(lg,1))) & (P - 1).
struct SideHash {
    uint64_t a, b;
    uint32_t shift, mask;
};

struct HashPair {
    SideHash ha, hb;
};

__host__ __device__ __forceinline__ uint32_t side_hash(const SideHash &h, uint32_t x) {
    return (uint32_t)((h.a * (uint64_t)x + h.b) >> h.shift) & h.mask;
}

__host__ __device__ __forceinline__ uint32_t partition_hash(const HashPair &hp, uint32_t i,
                                                            uint32_t j) {
    return (side_hash(hp.ha, i) + side_hash(hp.hb, j)) & hp.ha.mask;
}

// Count-Sketch sign of entry (i,j) (Preliminaries, "Count-Sketch"):
// s(i,j) = s_a(i) s_b(j), each side's sign taken from the top bit of a
// multiply-add hash ((c x + d) mod 2^64) whose (c, d) are the third and
// fourth SplitMix64 outputs of that side's seed.  The product of the two
// signs is negative exactly when the two top bits differ.
struct SignPair {
    uint64_t ca, da, cb, db;
};

__host__ __device__ __forceinline__ bool sign_negative(const SignPair &s, uint32_t i,
                                                       uint32_t j) {
    return ((s.ca * (uint64_t)i + s.da) ^ (s.cb * (uint64_t)j + s.db)) >> 63;
}

// Slot position hash inside one partition table (independent of the
// partition hash): the 64-bit finaliser of MurmurHash3 (Appleby).
__host__ __device__ __forceinline__ uint64_t slot_mix(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

__host__ __device__ __forceinline__ uint64_t make_key(uint32_t i, uint32_t j) {
    return ((uint64_t)i << 32) | j;
}

// A 16-byte exact-table slot: the key, then an int32 count (int mode) or an
// fp64 sum (real mode) in the second word.
struct __align__(16) Slot {
    unsigned long long key;
    unsigned long long val;  // u32 count in the low half, or the bits of a double
};

// Device-side counters and the status word of one plan.
struct DevCounters {
    unsigned int status;
    unsigned int work_next;          // dynamic work-item counter
    unsigned long long terms;        // terms enumerated
    unsigned long long flushed;      // entries flushed from on-chip tables
    unsigned long long spill_n;      // spilled updates
    unsigned long long bad_index;    // first bad index seen (debug checks)
    unsigned int long_n;             // long vectors deferred by the sorter
    unsigned int pad;
    unsigned long long work64;       // 64-bit work-item counter (batched launch)
};

struct SpillRec {
    unsigned long long key;
    unsigned long long val;
};

// Everything a table-update kernel needs to reach the partition tables.
// Every field has a default, so a view built field by field never carries
// garbage into the update paths.
struct TableView {
    Slot *slots = nullptr;
    const unsigned long long *part_off = nullptr;   // first slot of each partition
    const unsigned long long *part_mask = nullptr;  // capacity - 1 (a power of two)
    unsigned int *part_full = nullptr;              // set once a partition had no free slot
    SpillRec *spill = nullptr;
    unsigned long long spill_cap = 0;
    DevCounters *dc = nullptr;
    int value_type = 0;
    int keep_in_l2 = 0;                       // bucket loads hint evict-last (routed apply)
    // summary mode (Space-Saving semantics per partition)
    int summary = 0;                          // 1: tables are counter summaries;
                                              // 2: one locked bucket of bucket_ell
                                              //    counters per partition
    unsigned int *locks = nullptr;            // summary 2: a ticket lock per partition
                                              //    (next ticket, now serving)
    long long lock_wait = 8ll << 30;          // summary 2: SM-clock cycles a waiter
                                              //    waits for a lock before giving up
    uint32_t bucket_ell = 0;
    unsigned int *live = nullptr;             // occupied slots per partition
    const unsigned int *floor = nullptr;      // current floor (min count) per partition
    unsigned int hard_cap = 0;                // max live slots before new keys spill
    // reserved exact counters probed before the summaries (0 slots = none)
    unsigned long long res_off = 0, res_mask = 0;  // [res_off, res_off + res_mask + 1)
    int has_reserved = 0;
    // items that occur in a reserved key (bit per index): other pairs skip the probe
    const unsigned int *res_bits_a = nullptr, *res_bits_b = nullptr;
};

struct AccumulateArgs {
    // inputs
    const int64_t *a_ptr;
    const int32_t *a_idx;
    const float *a_val;
    const int64_t *b_ptr;
    const int32_t *b_idx;      // b indices in stream order, or sorted by h_b
    const float *b_val;
    int64_t K;
    int32_t n_rows, n_cols;
    // work decomposition
    uint32_t groups;           // G; group g covers partitions [g P/G, (g+1) P/G)
    uint32_t group_begin, group_end;
    uint32_t tile;             // outer products per work item
    uint32_t n_tiles;
    int mode;                  // CRP_FULL | CRP_UPPER
    int use_match;
    int debug_checks;
    int direct;                // no on-chip table (CRP_PLAN_DIRECT)
    uint32_t smem_slots;       // power of two
    HashPair hp;
    TableView tv;
    // hot block: exact dense counters for pairs of frequent items (direct,
    // int mode); rank arrays hold the item's row/column in the block or
    // 0xFFFF
    const uint16_t *hot_rank_a = nullptr;
    const uint16_t *hot_rank_b = nullptr;
    unsigned int *hot_block = nullptr;
    uint32_t hot_R = 0;
    // ragged block of reserved pairs (summary mode; hot_block then holds its
    // cells): row r = hot_rank_a has resv_len[r] cells from resv_off[r],
    // indexed by hot_rank_b; a cell holding kCellOff is not reserved (its
    // pair takes the summary path)
    const unsigned int *resv_len = nullptr, *resv_off = nullptr;
    // warm stripes: dense counters for the pairs (warm row, any column) and
    // (any row, warm column) outside the hot block
    const uint16_t *warm_rank_a = nullptr;
    const uint16_t *warm_rank_b = nullptr;
    unsigned int *warm_a = nullptr;   // [warm_W][n_cols]
    unsigned int *warm_b = nullptr;   // [warm_W][n_rows]
    uint32_t warm_W = 0;
    // the warm items are the first warm_W hot ranks (warm rank == hot rank)
    int warm_in_hot = 0;
    // interval [part_lo, part_hi) of partitions kept (Figure 1, CRoP on [q, r))
    uint32_t part_lo = 0, part_hi = 0xFFFFFFFFu;
    // pairs i < j of T^T T with a_k == b_k (same sorted list): the window of
    // the a entry at position x starts at position x + 1 of b_k
    int sym_upper = 0;
    // Count-Sketch: P estimators, int64 (int mode) or fp64 (real mode);
    // sketch_smem > 0 (direct kernel): each CTA sums into that many copies
    // of the estimators in shared memory and adds them at the end
    void *sketch = nullptr;
    SignPair sg = {0, 0, 0, 0};
    uint32_t sketch_smem = 0;
};

// Count-Sketch estimates from t <= kSketchMaxT plans (crp_sketch.cu)
constexpr int kSketchMaxT = 32;
struct SketchSet {
    HashPair hp[kSketchMaxT];
    SignPair sg[kSketchMaxT];
    const void *cs[kSketchMaxT];
    int32_t t;
    int32_t value_type;
};
cudaError_t launch_sketch_estimate(const SketchSet &S, const int32_t *i, const int32_t *j,
                                   int64_t n, int32_t n_rows, int32_t n_cols, double *out,
                                   unsigned int *bad, cudaStream_t s);
// the direct kernel keeps its sketch in shared memory for P <= 4096, in
// 4096 / P copies (at most one per warp): 32 KB per CTA
constexpr uint32_t kSketchSmemMaxP = 4096;

// Two-phase (routed) accumulation: bins of records per partition group.
constexpr uint32_t kChunkRecs = 512;   // records per chunk of the routed pool
struct RouteArgs {
    AccumulateArgs acc;        // enumeration inputs, hash and table view
    void *pool;                // n_chunks chunks of kChunkRecs records: u64 keys (int)
                               // or {key, p, e} (real); unused tails hold kEmptyKey
    unsigned int *chunk_bin;   // bin of each installed chunk, ~0u for none
    unsigned int *chunk_next;  // chunks handed out (may pass n_chunks)
    unsigned int *order;       // installed chunk ids grouped by bin
    unsigned int *start;       // B + 1: first entry of each bin in order[]
    uint32_t n_chunks;
    uint32_t B, B_shift;
    uint32_t core_H;           // ranks < core_H of the hot block count in shared memory first
    unsigned int *ov_next;     // records in the overflow chunks (chunks [0, ov_cap / kChunkRecs))
    uint32_t ov_cap;
};
cudaError_t launch_route(const RouteArgs &RA, int grid, cudaStream_t s);
// Records the routing phase will append: per outer product, the terms outside
// the dense tiers (hot pairs, warm rows, warm columns), summed into *out.
cudaError_t launch_count_records(const AccumulateArgs &A, unsigned long long *out,
                                 cudaStream_t s);
cudaError_t launch_apply(const RouteArgs &RA, unsigned int *count, unsigned int *fill, int grid,
                         cudaStream_t s);
size_t route_smem_bytes(uint32_t B, uint32_t core_H);

// Summary mode (crp_summary.cu)
cudaError_t launch_summary_compact(Slot *slots, const unsigned long long *part_off,
                                   const unsigned long long *part_mask, unsigned int *live,
                                   unsigned int *floor, const unsigned int *todo, uint32_t n_todo,
                                   uint32_t ell, uint32_t trigger, Slot *tmp, int grid,
                                   cudaStream_t s);
cudaError_t launch_reserve_bits(const unsigned long long *keys, int32_t n, unsigned int *bits_a,
                                unsigned int *bits_b, cudaStream_t s);
cudaError_t launch_reserve_insert(Slot *slots, unsigned long long res_off,
                                  unsigned long long res_mask, const unsigned long long *keys,
                                  int32_t n, cudaStream_t s);

// Hot block (crp_accumulate.cu)
cudaError_t launch_hot_flush(unsigned int *hot, uint32_t R, const int64_t *items_a,
                             const int64_t *items_b, HashPair hp, TableView tv,
                             unsigned long long *flushed, cudaStream_t s);
// The ragged reserved block: every cell kCellOff, then the reserved cells
// (indices cells[0, n)) 0; and its flush into the tables (clearing counts).
cudaError_t launch_reserve_cells(const unsigned int *cells, int32_t n, unsigned int *block,
                                 uint64_t n_cells, cudaStream_t s);
cudaError_t launch_reserve_flush(unsigned int *block, uint64_t n_cells, const unsigned int *res_off,
                                 uint32_t rows, const int64_t *items_a, const int64_t *items_b,
                                 HashPair hp, TableView tv, unsigned long long *flushed,
                                 cudaStream_t s);
cudaError_t launch_hot_ranks(uint16_t *rank, int32_t n, const int64_t *items, uint32_t R,
                             cudaStream_t s);
cudaError_t launch_warm_flush(unsigned int *stripe, uint32_t W, int32_t n_other,
                              const int64_t *items, int rows, HashPair hp, TableView tv,
                              unsigned long long *flushed, cudaStream_t s);

// Selections (crp_select.cu)
int select_grid_for(int64_t n);
cudaError_t order_by_count(int64_t *items, const unsigned int *cnt, uint32_t R, cudaStream_t s);
// kernels one select_top call launches (four histogram passes, four digit
// picks, the emit)
constexpr int kSelectTopLaunches = 9;
cudaError_t select_top(const uint32_t *key, int64_t n, int64_t K, int64_t *out,
                       unsigned int *scratch /* 260 */, cudaStream_t s);
cudaError_t launch_item_counts(const int32_t *idx, int64_t nnz, int32_t n_items, unsigned int *cnt,
                               cudaStream_t s);
cudaError_t launch_item_counts_at(const int32_t *idx, const int64_t *nnz_at, int64_t nnz_hint,
                                  int32_t n_items, unsigned int *cnt, cudaStream_t s);

// Record the calling thread's error message (read by crp_last_error).
void set_last_error(const std::string &msg);

// Launchers (defined in the .cu files).
cudaError_t launch_sort_by_hash(const int64_t *ptr, const int32_t *idx, const float *val,
                                int64_t K, SideHash h, int32_t *out_idx, float *out_val,
                                uint32_t *out_hash, DevCounters *dc, unsigned int *long_list,
                                int sm_count, cudaStream_t s);
cudaError_t launch_accumulate(const AccumulateArgs &args, const uint32_t *b_hash, int grid,
                              cudaStream_t s);
int accumulate_block_threads();
int accumulate_max_blocks_per_sm(int value_type, uint32_t smem_slots, bool direct);
size_t accumulate_smem_bytes(int value_type, uint32_t smem_slots);
cudaError_t launch_count_terms(const int64_t *a_ptr, const int64_t *b_ptr, int64_t K,
                               unsigned long long *out, cudaStream_t s);
cudaError_t launch_fill_empty(Slot *slots, uint64_t n, cudaStream_t s);
cudaError_t launch_partition_sums(const Slot *slots, const unsigned long long *part_off,
                                  const unsigned long long *part_mask, uint32_t P,
                                  int value_type, unsigned long long *terms_out,
                                  unsigned long long *live_out, cudaStream_t s);
cudaError_t launch_spill_reinsert(const SpillRec *spill, uint64_t n, HashPair hp,
                                  TableView tv, cudaStream_t s);
cudaError_t launch_rehash_partition(const Slot *old_slots, uint64_t old_off, uint64_t old_cap,
                                    TableView tv, uint64_t new_off, uint64_t new_mask,
                                    cudaStream_t s);
cudaError_t launch_validate_sparse(const int64_t *ptr, const int32_t *idx, int64_t K, int64_t nnz,
                                   int32_t n_minor, unsigned int *bad, cudaStream_t s);

// Top-k (crp_topk.cu)
struct TopkCand {
    unsigned long long wkey;  // order-preserving bits of |w| (larger = heavier)
    unsigned long long ij;    // (i << 32) | j
    double w;
    double wl;
};
cudaError_t launch_topk_hist(const Slot *slots, uint64_t n, int value_type, int upper_only,
                             int sample_shift, unsigned int *hist, cudaStream_t s);
cudaError_t launch_topk_collect(const Slot *slots, uint64_t n, int value_type, int upper_only,
                                unsigned int bucket_lo, TopkCand *out, unsigned int *count,
                                unsigned int cap, cudaStream_t s);
cudaError_t launch_cand_hist(const TopkCand *c, unsigned int n, unsigned int *hist,
                             cudaStream_t s);
cudaError_t launch_cand_collect(const TopkCand *c, unsigned int n, unsigned int b_lo,
                                TopkCand *out, unsigned int *cnt, cudaStream_t s);
cudaError_t launch_topk_digit_hist(const TopkCand *c, unsigned int n, int digit,
                                   unsigned int *hist, cudaStream_t s);
cudaError_t launch_topk_digit_split(const TopkCand *c, unsigned int n, int digit,
                                    unsigned int pivot, TopkCand *sel, unsigned int *sel_n,
                                    TopkCand *keep, unsigned int *keep_n, cudaStream_t s);
// Sort n candidates (n <= kTopkSortMax) and write the first n_write.
cudaError_t launch_topk_sort_write(const TopkCand *c, unsigned int n, unsigned int n_write,
                                   int32_t *i_out, int32_t *j_out, double *w_out, double *wl_out,
                                   cudaStream_t s);
cudaError_t launch_export_range(const Slot *slots, const unsigned long long *part_off,
                                const unsigned long long *part_mask, uint32_t p0, uint32_t p1,
                                const unsigned long long *base, int value_type, int32_t *i_out,
                                int32_t *j_out, double *w_out, double *wl_out, cudaStream_t s);
unsigned int topk_bucket_host(unsigned long long wkey);
constexpr int kTopkBuckets = 4096;
constexpr int kTopkSortMax = 8192;

}  // namespace crp
