/*
 * crp.h -- C ABI of the column-row partitioned sparse product on GB300.
 *
 * The library computes C = A B as the sum of outer products of the columns
 * of A and the rows of B (the column-row method; paper "On Parallelizing
 * Matrix Multiplication by the Column-Row Method", Campagna, Kutzkov, Pagh:
 * Preliminaries, Notation: the weight of entry (i,j) is sum_k a_k(i) b_k(j)).
 * Every output entry (i,j) belongs to exactly one of P hash partitions,
 *     h(i,j) = (h_a(i) + h_b(j)) mod P                      (Section 4, Lemma 1)
 * whatever the structure of the outer product it appears in, so partitions
 * are accumulated independently (Section 4, "Our approach": CRoP).  Each
 * partition holds either an exact table of its entries or a counter summary
 * with Space-Saving guarantees (Preliminaries; Figure 1).
 *
 * Conventions for every call below:
 *  - Indices are 0-based ([n] = {0..n-1}, Preliminaries).
 *  - "device" pointers are CUDA device (or managed) memory of the device that
 *    was current at crp_plan_create; "host or device" pointers are detected
 *    with cudaPointerGetAttributes.
 *  - The caller owns every buffer it passes; the plan owns its tables,
 *    summaries and scratch, which crp_plan_destroy frees.
 *  - Work is enqueued on the plan's stream and is asynchronous; errors the
 *    host can see are returned at once, errors the device records (a full
 *    table, an index out of range) are returned by crp_sync.
 *  - No call throws, traps or aborts.  A plan is not thread-safe.
 *  - crp_last_error() returns a message for the calling thread's last error.
 *
 * Hash family (a reading: the paper only requires pairwise independent
 * h_a, h_b, Lemma 1).  With s = seed_a (resp. seed_b), (a, b) are the first
 * two outputs of SplitMix64 started from state s, and for a 32-bit index x
 *     h(x) = ((a*x + b) mod 2^64) >> (64 - log2 P)     (multiply-add-shift)
 * P must be a power of two; P = 1 puts everything in partition 0.
 */
#ifndef CRP_H
#define CRP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CRP_OK = 0,
    CRP_EINVAL = 1,          /* bad argument or descriptor */
    CRP_ENOMEM = 2,          /* device allocation failed */
    CRP_ETABLE_FULL = 3,     /* a partition table ran out of slots and the
                                entries could not be kept */
    CRP_ETIMEOUT = 4,        /* a bounded device wait gave up */
    CRP_ECUDA = 5,           /* CUDA runtime error (message in last_error) */
    CRP_EUNSUPPORTED = 6     /* valid but outside what this build handles */
} crp_status;

/* value_type */
enum { CRP_I32 = 0,          /* {0,1} inputs (val == NULL), exact int32 counts */
       CRP_F32_COMP = 1 };   /* fp32 inputs; each term is the exact product
                                p + e (fp32 TwoProduct); the on-chip-table
                                variant sums an entry's terms per CTA as a
                                compensated fp32 pair (TwoSum) and adds the
                                pair to the fp64 entry at its flush; the
                                direct and routed variants add each p + e
                                (exact in fp64) to the fp64 entry with an
                                atomic.  fp64 per-entry result. */
/* mode */
enum { CRP_FULL = 0,         /* every entry (i,j) */
       CRP_UPPER = 1 };      /* only i < j: pairs above the diagonal, the
                                frequent-pair view of T^T T (Section 6) */
/* crp_topk flags */
enum { CRP_TOPK_UPPER = 1 }; /* report only i < j */
/* crp_plan_desc.flags */
enum { CRP_PLAN_NO_WARP_MATCH = 1,  /* skip __match_any_sync pre-combining */
       CRP_PLAN_DEBUG_CHECKS = 2,   /* validate inputs and bounds-check indices */
       CRP_PLAN_DIRECT = 4,         /* no on-chip combining table: every
                                       (warp-combined) term updates its
                                       partition table in HBM directly */
       CRP_PLAN_SORTED_ROWS = 16,   /* the caller guarantees every vector's
                                       indices are distinct and ascending: with
                                       CRP_UPPER and A, B the same arrays (T^T T)
                                       only the pairs i < j are enumerated */
       CRP_PLAN_SKETCH = 32,        /* also keep a Count-Sketch with one
                                       estimator per partition (Preliminaries
                                       and Figure 1: CS[h(e)] += e s(e) for
                                       every term e), updated in the same pass
                                       as the tables (per term in direct
                                       plans, per combined entry when the
                                       on-chip table flushes; the sketch is
                                       linear, so both give the same sums).
                                       Not with CRP_PLAN_ROUTED; see
                                       crp_sketch_read. */
       CRP_PLAN_LOCKED_SUMMARY = 64,/* summary plans: each partition is ONE
                                       Space-Saving summary of exactly
                                       summary_counters (<= 64) counters, a
                                       bucket updated under its own lock in
                                       the order updates arrive -- the
                                       sequential algorithm of the
                                       Preliminaries on one arrival order of
                                       the partition's terms; one enumeration
                                       launch per call, no compaction.  The
                                       paper's regime of many small buckets
                                       (Section 6: 10^6 buckets, 2 counters).
                                       By default each CTA first combines
                                       equal keys in its on-chip table and
                                       flushes weighted updates (heavy pairs
                                       then take few locks); with
                                       CRP_PLAN_DIRECT every warp-combined
                                       term takes its bucket's lock, and
                                       hot_items / warm_items may be set (the
                                       dense tiers count pairs of frequent
                                       items exactly and add them as weighted
                                       updates at the end of the call).
                                       reserved_counters may not be set. */
       CRP_PLAN_ROUTED = 8 };       /* two phases: enumerate every term once
                                       into per-partition-group bins, then
                                       apply the bins group by group so each
                                       group's table region stays in L2
                                       (bins = `groups` when set, else sized
                                       to ~48 MB of table per group) */

/* A compressed sparse matrix viewed as K vectors: vector k holds indices
 * idx[ptr[k] .. ptr[k+1]) (each < n_minor, distinct within a vector) with
 * values val[...] (val == NULL: all ones).  A is passed compressed by column
 * (CSC: vector k = column a_k, indices i) and B compressed by row (CSR:
 * vector k = row b_k, indices j); the paper stores A as column-major and B
 * as row-major triples (Section 4, "The algorithm").  For co-occurrence
 * counts T^T T of a transaction matrix T (CSR, rows = transactions) pass the
 * same CSR of T as both A and B (Section 6).  ptr, idx, val: device. */
typedef struct {
    int64_t n_major;        /* K, the number of vectors */
    int32_t n_minor;        /* index range */
    int32_t _pad;
    int64_t nnz;            /* ptr[n_major] */
    const int64_t *ptr;     /* device, n_major + 1 entries, ptr[0] == 0 */
    const int32_t *idx;     /* device, nnz entries */
    const float *val;       /* device, nnz entries, or NULL */
} crp_sparse;

typedef struct {
    int32_t n_rows, n_cols;       /* C is n_rows x n_cols */
    uint32_t P;                   /* partitions (power of two, >= 1), or 0:
                                     chosen, with groups, tile_vectors,
                                     smem_slots, the variant flags and the
                                     dense tiers, by crp_autotune on the first
                                     min(K, 2^21) outer products of the first
                                     crp_outer_accumulate (which then
                                     synchronises); exact plans over all
                                     partitions only */
    uint32_t _pad0;
    uint64_t seed_a, seed_b;      /* hash seeds of h_a and h_b */
    int32_t value_type;           /* CRP_I32 | CRP_F32_COMP */
    int32_t mode;                 /* CRP_FULL | CRP_UPPER */
    uint32_t summary_counters;    /* 0: exact tables; else counters per
                                     partition of a Space-Saving summary */
    uint32_t reserved_counters;   /* summary mode: exact counters for keys
                                     registered with crp_reserve (0 = none) */
    uint64_t table_capacity_hint; /* total exact-table slots wanted (0: the
                                     library sizes from the input of the first
                                     crp_outer_accumulate) */
    int32_t auto_grow;            /* exact mode: on a full partition keep the
                                     overflow in a spill list and grow that
                                     partition at crp_sync */
    uint32_t groups;              /* partition groups G (passes over the input;
                                     one CTA work item covers P/G partitions);
                                     0 = default */
    uint32_t tile_vectors;        /* outer products per work item; 0 = default */
    uint32_t smem_slots;          /* on-chip combining table slots per CTA
                                     (power of two); 0 = default */
    uint32_t flags;               /* CRP_PLAN_* */
    uint32_t hot_items;           /* CRP_PLAN_DIRECT or CRP_PLAN_ROUTED with
                                     CRP_I32 only: R > 0
                                     keeps exact dense counters (R x R, in L2)
                                     for the pairs of the R most frequent rows
                                     and columns, chosen per call from the
                                     first 1/64 of the outer products; their
                                     counts are added to the partition tables
                                     at the end of the call.  R <= 4096. */
    uint32_t target_load_pct;     /* exact tables sized by the library: at most
                                     this % of a partition's slots occupied per
                                     the estimate (0 = 65; <= 90) */
    uint32_t part_begin, part_end;/* the plan's interval [q, r) of partitions
                                     (Figure 1, CRoP run on one interval;
                                     Theorem 1's K instances use disjoint equal
                                     intervals): only entries with h(i,j) in it
                                     are accumulated and stored.  0, 0 = all.
                                     Exact mode only. */
    uint32_t warm_items;          /* CRP_PLAN_DIRECT or CRP_PLAN_ROUTED with
                                     CRP_I32 only: W > 0 keeps exact dense
                                     counters for every pair whose row (or
                                     else column) is among the W most frequent
                                     (W x n_cols and W x n_rows, in L2),
                                     after the hot block; W is lowered so the
                                     stripes fit 64 MB.  Same selection and
                                     flush as hot_items. */
    uint32_t route_pool_chunks;   /* CRP_PLAN_ROUTED: at most this many record
                                     chunks (512 records each) in the pool,
                                     overflow chunks included (0: sized from
                                     each call's count of routed records).  A
                                     pool too small for the records sends the
                                     rest to the overflow chunks and, once
                                     those fill, straight to the tables:
                                     slower, the same result.  For exercising
                                     those paths; no paper counterpart. */
    uint32_t lock_wait_us;        /* CRP_PLAN_LOCKED_SUMMARY: how long a warp
                                     waits for a bucket's lock, in
                                     microseconds of SM clock at 2 GHz, before
                                     it drops the update and the call reports
                                     CRP_ETIMEOUT (0: about 4 s) */
} crp_plan_desc;

typedef struct crp_plan crp_plan;

typedef struct {
    uint64_t terms;               /* outer-product terms enumerated */
    uint64_t flushed_updates;     /* on-chip entries flushed to partition
                                     tables (terms / this = combining ratio) */
    uint64_t entries;             /* live entries in all partitions */
    uint64_t table_slots;         /* allocated exact-table slots */
    uint64_t spilled;             /* updates held in the spill list */
    uint32_t full_partitions;     /* partitions that ran out of slots */
    uint32_t P;
    double max_over_mean_terms;   /* largest / mean per-partition terms (int
                                     mode; Theorem 1, Table 4) */
    double last_accumulate_ms;    /* device time of the last enumeration /
                                     combining kernel (CUDA events on the
                                     plan's stream) */
    uint64_t launches;            /* kernels this plan has launched */
    double last_route_ms;         /* routed mode: device time of the routing
                                     phase within last_accumulate_ms */
    uint64_t estimated_entries;   /* the nonzero entries of A B estimated
                                     before the tables were sized (distinct
                                     entries of one sampled partition group,
                                     times the number of groups; Section 4,
                                     "Parameters": estimating the size of the
                                     output); 0 when not sampled */
} crp_stats_t;

/* Create a plan: validates desc, derives the hash parameters and allocates
 * the partition tables (exact mode) or summaries (summary mode) on the
 * current device.  The P partitions are the paper's hash buckets, h the
 * pairwise independent h(i,j) = (h_a(i) + h_b(j)) mod P of Lemma 1, and the
 * choice of P, like the paper's number of buckets, is a tuning parameter
 * (Section 4, "Parameters"; P = 0 tunes it).  stream: a cudaStream_t (NULL = legacy default stream).
 * Returns CRP_EINVAL for a P that is not a power of two, n_rows/n_cols <= 0,
 * an unknown value_type/mode, or smem_slots not a power of two. */
crp_status crp_plan_create(crp_plan **out, const crp_plan_desc *desc, void *stream);

/* Free everything the plan owns (NULL is accepted). */
void crp_plan_destroy(crp_plan *plan);

/* Zero all partition tables / summaries and statistics (capacity is kept). */
crp_status crp_reset(crp_plan *plan);

/* Add sum_k a_k b_k over the K outer products of A (CSC) and B (CSR) into
 * the partition tables (Figure 1, CRoP: for each k hash every entry of a_k
 * b_k to its partition and update that partition's table or summary).
 * Additive across calls, so a stream is processed in chunks of k.
 * A->n_major must equal B->n_major, A->n_minor == n_rows, B->n_minor ==
 * n_cols.  CRP_I32 requires A->val == B->val == NULL.  In CRP_UPPER mode
 * only terms with i < j are added.  Asynchronous: a full table or a bad index
 * is reported by crp_sync. */
crp_status crp_outer_accumulate(crp_plan *plan, const crp_sparse *A_csc, const crp_sparse *B_csr);

/* Wait for the plan's stream and return the status the device recorded --
 * the end of one CRoP pass over the input (Figure 1), after which every
 * partition holds its entries -- (CRP_ETABLE_FULL, CRP_EINVAL for an index
 * >= n_minor when
 * CRP_PLAN_DEBUG_CHECKS is set, CRP_ETIMEOUT).  With auto_grow, full
 * partitions are grown and their spilled updates re-inserted first. */
crp_status crp_sync(crp_plan *plan);

/* The k heaviest entries (largest |weight|; ties by i then j ascending): the
 * query the paper's case study answers, the most frequent pairs of items
 * (Section 6; in summary mode the entries the summaries guarantee,
 * Preliminaries),
 * written in that order to i_out, j_out, w_out (host or device, k entries
 * each); w_lower (nullable) receives the lower bound in summary mode and the
 * weight itself in exact mode.  *n_out (host) = entries written (< k when C
 * has fewer nonzero entries).  flags: CRP_TOPK_UPPER.  1 <= k <= 8192.
 * Synchronises the plan's stream. */
crp_status crp_topk(crp_plan *plan, int32_t k, uint32_t flags, int32_t *i_out, int32_t *j_out,
                    double *w_out, double *w_lower, int32_t *n_out);

/* How many crp_topk calls of the plan were answered from the hot block alone.
 * For CRP_I32 exact plans with hot_items > 0 the plan keeps the degree of
 * every row and column over the calls since the last reset (deg(i) = number
 * of outer products whose a_k holds i; deg(j) likewise in B).  An entry is at
 * most min(deg(i), deg(j)), so when the k-th heaviest of the hot pairs
 * (hot rows x hot columns of the last call) weighs more than every degree
 * outside the hot set, no other entry can be in the top k and crp_topk
 * answers from the hot pairs without scanning the tables; otherwise it scans
 * them.  The result is the same either way. */
uint64_t crp_topk_certified_calls(const crp_plan *plan);

/* Summary mode (desc.summary_counters = ell > 0, CRP_I32 only): each
 * partition keeps a counter summary with the Space-Saving guarantees of the
 * paper's Preliminaries -- for every key of partition p with stream weight
 * W_p: lower <= true <= upper, upper - lower <= W_p / ell, and every key with
 * true weight > W_p / ell is recorded; after each crp_outer_accumulate a
 * partition holds at most ell keys.  crp_topk then ranks by the upper bound
 * and reports the lower bound in w_lower; crp_export_partitions gives both.
 *
 * crp_reserve registers keys ((uint64_t)i << 32 | j; host or device array
 * of n) whose updates go to exact counters instead of the summaries
 * (desc.reserved_counters bounds their number).  During accumulation they
 * are counted in a ragged block over their rows and columns (device memory
 * about the number of reserved keys when they cluster on few rows and
 * columns; more than 64 Mi cells, or 65,535 distinct rows or columns, fall
 * back to a hash probe of the exact counters) and added to the exact
 * counters at the end of each call.  Reserve before the accumulate calls
 * whose terms should be counted exactly: weight added to a key before it was
 * reserved stays in its partition's summary.  crp_reset keeps the reserved
 * keys and zeroes their counts.  Synchronises. */
crp_status crp_reserve(crp_plan *plan, const uint64_t *keys, int32_t n);

/* Test hook for the bounded lock wait of locked-bucket plans
 * (CRP_PLAN_LOCKED_SUMMARY); the paper has no counterpart.  Takes partition
 * p's bucket lock on behalf of the host and never hands it on (the next
 * ticket is advanced on the device, stream-ordered): every later update of
 * p waits lock_wait_us, gives up, and crp_sync returns CRP_ETIMEOUT; other
 * waiters of the plan give up at once after the first timeout.  crp_reset
 * releases it.  CRP_EINVAL for other plans or p >= P. */
crp_status crp_debug_hold_lock(crp_plan *plan, uint32_t p);

/* Partition of entry (i,j): (h_a(i) + h_b(j)) mod P, computed on the host. */
uint32_t crp_partition_of(const crp_plan *plan, int32_t i, int32_t j);

/* Copy the entries of partitions [p_begin, p_end) to i_out, j_out, w_out
 * (and w_lower, nullable; host or device; `capacity` entries each), grouped
 * by partition in ascending order, unordered within a partition.  *n_out =
 * number of entries in those partitions, even when it exceeds capacity (then
 * nothing is written and CRP_EINVAL is returned).  Synchronises. */
crp_status crp_export_partitions(crp_plan *plan, uint32_t p_begin, uint32_t p_end, int32_t *i_out,
                                 int32_t *j_out, double *w_out, double *w_lower,
                                 int64_t capacity, int64_t *n_out);

/* Per-partition term counts (int mode: sum of the counts in the partition)
 * into terms_out (host, P entries, nullable) and aggregate statistics into
 * *stats.  Synchronises. */
crp_status crp_stats(crp_plan *plan, crp_stats_t *stats, uint64_t *terms_out);

/* Device time of the last enumeration kernel launched by crp_outer_accumulate
 * (CUDA events on the plan's stream; waits for that kernel) and the number of
 * kernels the plan has launched so far.  Either pointer may be NULL.  Cheap:
 * it does not scan the tables. */
crp_status crp_timing(crp_plan *plan, double *accumulate_ms, uint64_t *launches);

/* Count-Sketch of a plan created with CRP_PLAN_SKETCH (Preliminaries,
 * "Count-Sketch"; Figure 1 updates CS[h(e)] by e s(e) for every term e of
 * every outer product, h the plan's partition hash).  The sign of entry
 * (i,j) is s(i,j) = s_a(i) s_b(j), s_x(v) = +1 or -1 from the top bit of
 * (c v + d) mod 2^64 with (c, d) the third and fourth SplitMix64 outputs of
 * that side's seed (the first two give h_x).  The sketch adds up over the
 * plan's accumulate calls; crp_reset zeroes it.
 *
 * crp_sketch_read copies the P estimators to out (host or device): int64
 * for CRP_I32 plans (exact), double for CRP_F32_COMP plans (each term the
 * exact fp32 product, summed in fp64 in no fixed order).  Synchronises.
 * CRP_EINVAL when the plan keeps no sketch. */
crp_status crp_sketch_read(crp_plan *plan, void *out);

/* Estimates of entries (i[q], j[q]), q < n, from t plans (1 <= t <= 32) with
 * sketches, the same P, n_rows, n_cols and value type and independent seeds:
 * plan r's estimate is s_r(i,j) CS_r[h_r(i,j)], and out[q] is the median of
 * the t estimates (the mean of the two middle ones when t is even), the
 * paper's median over independent runs.  i, j (int32) and out (double, n
 * entries) are device arrays; indices must lie in [0, n_rows) and [0, n_cols)
 * (CRP_EINVAL otherwise; the check costs one small readback).  Runs on
 * plans[0]'s stream after every plan's pending work; synchronises. */
crp_status crp_sketch_estimate(crp_plan *const *plans, int32_t t, const int32_t *i,
                               const int32_t *j, int64_t n, double *out);

/* Measurement helper, not on the product path: device time (*ms_out) of
 * n_updates random updates into a freshly allocated region of region_bytes
 * (a power of two >= 4096; allocated and freed inside, default stream).
 * mode 0: 32-bit atomic adds without return value at random words; mode 1:
 * the exact-table update (read key, CAS an empty 16-byte slot, 32-bit add)
 * with keys drawn from region/32 distinct values.  Gives the empirical update
 * rate of an L2-resident vs an HBM-resident table.  Synchronises. */
crp_status crp_probe_update_rate(uint64_t region_bytes, uint64_t n_updates, int mode,
                                 double *ms_out);

/* An exact product for callers that cannot allocate device memory.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- code running under an external memory manager that owns
 * the device, code in a region where an allocation would synchronise or is
 * forbidden, plug-ins whose host forbids the CUDA allocator.  It computes the
 * same entries as crp_plan_create + crp_outer_accumulate + crp_export_partitions
 * (desc fields n_rows, n_cols, P, seeds, value_type, mode are used; the rest
 * are ignored) but keeps its partition tables in a file-scope static device
 * array of 2^20 16-byte slots (16 MiB, held by every device that loads the
 * library until the process exits) split evenly over P <= 1024 partitions.
 * It calls no cudaMalloc, cudaFree or allocating library routine.
 *   A, B: device inputs as for crp_outer_accumulate.
 *   i_out, j_out, w_out: device arrays of `capacity` entries (caller-owned);
 *     the entries are written unordered.  *n_out (host) = number of nonzero
 *     entries, also when it exceeds capacity (then CRP_EINVAL and nothing
 *     beyond capacity is written).
 *   stream: a cudaStream_t; the call synchronises it before returning.
 * Errors: CRP_EINVAL for P > 1024 or not a power of two, mismatched shapes or
 * a too small output; CRP_ETABLE_FULL when a partition of the static table
 * overflows (the product has too many entries for this entry point; the
 * updates that met the full partition are lost, so *n_out is set to 0 and
 * the output arrays hold no usable result).
 * The first call in a CUDA context (per device: the primary context, or one
 * the caller made current) looks up the static array's device address with
 * cudaGetSymbolAddress, that device current, and keeps it for that context;
 * make that first call before any stream capture.  A call in another context
 * (after cudaDeviceReset, say) looks the address up again.  Every call
 * clears and reuses the same array, so calls whose work overlaps on the GPU
 * race: serialise them. */
crp_status crp_outer_product_noalloc(const crp_plan_desc *desc, const crp_sparse *A,
                                     const crp_sparse *B, int32_t *i_out, int32_t *j_out,
                                     double *w_out, int64_t capacity, int64_t *n_out,
                                     void *stream);

/* Batched products (many independent problems, one persistent launch).
 * Problem q computes A[q] B[q] (A[q] CSC, B[q] CSR, {0,1} values, device
 * pointers; A and B are HOST arrays of nprob descriptors) into its own P
 * partition tables; desc supplies P (<= 4096), seeds, mode and tile_vectors
 * (CRP_I32 only).  crp_batch_create counts each problem's terms, sizes its
 * tables from a sampling launch (terms of partitions [0, P/16) accumulated
 * exactly, distinct count scaled up; Section 4 "Parameters"), and captures
 * table reset + the persistent kernel into one CUDA graph on a private
 * stream.  All problems' work items (problem, tile of outer products) form a
 * single queue drained by that kernel.
 * desc->hot_items = R > 0 (at most 255; ignored with ready flags) adds a
 * dense tier per problem: each run counts the items of the problem's first
 * max(4096, K/64) outer products per side, takes the R most frequent of each
 * side, counts pairs of two of them in an R x R block instead of the tables,
 * and adds the block into the tables after the persistent kernel (results
 * unchanged; the graph holds these kernels too).
 * wait_timeout_ns > 0 enables per-problem ready flags (crp_batch_set_ready;
 * all start ready): a CTA that meets a problem whose flag is cleared waits at
 * most wait_timeout_ns, then skips it and crp_batch_sync returns
 * CRP_ETIMEOUT.  stream: where runs are launched (a cudaStream_t). */
typedef struct crp_batch crp_batch;
crp_status crp_batch_create(crp_batch **out, const crp_plan_desc *desc, int32_t nprob,
                            const crp_sparse *A, const crp_sparse *B, uint64_t wait_timeout_ns,
                            void *stream);
/* Launch the captured graph (reset every table, accumulate every problem). */
crp_status crp_batch_run(crp_batch *batch);
/* Wait; *ms (nullable) = device time of the last run, *terms (nullable) =
 * terms it enumerated.  Returns the recorded status (CRP_ETIMEOUT,
 * CRP_ETABLE_FULL). */
crp_status crp_batch_sync(crp_batch *batch, double *ms, uint64_t *terms);
/* Mark problem q's inputs ready (1) or withheld (0); synchronous copy. */
crp_status crp_batch_set_ready(crp_batch *batch, int32_t q, int32_t ready);
/* Entries of problem q (host or device outputs, `capacity` each; grouped by
 * partition); *n_out = entries, also when > capacity (then CRP_EINVAL). */
crp_status crp_batch_export(crp_batch *batch, int32_t q, int32_t *i_out, int32_t *j_out,
                            double *w_out, int64_t capacity, int64_t *n_out);
/* Total terms over all problems, allocated table slots, kernels launched. */
crp_status crp_batch_info(const crp_batch *batch, uint64_t *total_terms, uint64_t *table_slots,
                          uint64_t *launches);
void crp_batch_destroy(crp_batch *batch);

/* Heavy-pair predictor (not in the paper): a 2 -> 64 -> 64 -> 1 ReLU network
 * y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 whose two hidden products run on
 * the tcgen05 tensor cores (bf16 operands, fp32 accumulation in TMEM).
 * params: device fp32 array of crp_mlp_param_count() = 4417 values laid out as
 * W1[64][2], b1[64], W2[64][64], b2[64], w3[64], b3.  All pointers device;
 * every call synchronises `stream` (a cudaStream_t) and returns CRP_ETIMEOUT
 * if a bounded wait for tensor-core completion gave up. */
int32_t crp_mlp_param_count(void);
/* y[m] = network(x[2m], x[2m+1]) for m < n. */
crp_status crp_mlp_forward(const float *params, const float *x, float *y, int64_t n,
                           void *stream);
/* Mean squared error over n rows, L = sum_m (y_m - t_m)^2 / n_total, into
 * *loss, and dL/dparams into grad (4417 floats, overwritten).  The backward
 * products use bf16 operands (dZ2, dZ1, the saved activations). */
crp_status crp_mlp_grad(const float *params, const float *x, const float *t, int64_t n,
                        int64_t n_total, float *grad, float *loss, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8; step >= 1) on params with
 * moment buffers m, v (4417 floats each).  Asynchronous. */
crp_status crp_mlp_adam(float *params, float *m, float *v, const float *grad, float lr,
                        int32_t step, void *stream);
/* Candidate heavy pairs from a prefix of the stream: item counts c over the
 * prefix transactions (CSR, device), the R items of largest count, and every
 * pair i < j of them with features x = (log(1+c_i), log(1+c_j)) / log(1+max c).
 * Outputs (device, capacity >= R(R-1)/2): i_out, j_out, x_out (2 per pair). */
crp_status crp_candidate_pairs(const crp_sparse *prefix, int32_t n_items, int32_t R,
                               int32_t *i_out, int32_t *j_out, float *x_out, int64_t capacity,
                               int64_t *n_out, void *stream);
/* Score the candidate pairs with the network (params, device) or, when params
 * is NULL, with the product-of-marginals heuristic log(1+c_i) + log(1+c_j),
 * and crp_reserve the n_reserve best (both orders when full_mode != 0). */
crp_status crp_predict_reserve(crp_plan *plan, const crp_sparse *prefix, int32_t n_items,
                               const float *params, int32_t R, int32_t n_reserve,
                               int32_t full_mode, void *stream);

/* Launch-configuration autotuner.  Times candidate configurations of the exact
 * product -- P in {256, 1024, 4096}; the on-chip combining table (8192 or
 * 16384 slots), direct HBM updates (tiles of 32/64/256 outer products) or the
 * routed two-phase variant (128, 256 or size-derived bins); for CRP_I32 also
 * hot blocks of 1024 or 4096 items -- on the first sample_vectors outer products of
 * A and B (<= 0: all), with tables sized by the library's estimate, and
 * writes into *best a copy of *base with P, groups, tile_vectors, smem_slots
 * and the variant flags of the fastest (*best_terms_per_s, nullable, its
 * rate).  cache_path (nullable): a text file of previous results keyed by
 * device name and input shape class; a hit returns without timing, a miss
 * appends the new result.  Creates and destroys plans; synchronises. */
crp_status crp_autotune(const crp_plan_desc *base, const crp_sparse *A, const crp_sparse *B,
                        int64_t sample_vectors, const char *cache_path, crp_plan_desc *best,
                        double *best_terms_per_s, void *stream);

/* Autotuner of batched products (crp_batch_create): times the persistent
 * launch of a sample of the problems -- every (nprob / sample_probs)-th
 * problem, sample_probs <= 0 meaning all -- for P in {64, 256, 1024, 4096}
 * and tile_vectors in {16, 32, 64, 128}, then hot_items in {64, 128, 255} on the
 * fastest of those, and writes into *best a copy of *base with the fastest
 * P, tile_vectors and hot_items (*best_terms_per_s, nullable: its rate on
 * the sample).  The paper leaves the number of hash buckets and
 * the work per processor to tuning (Section 4, "Parameters"); this is that
 * choice made by measurement.  A, B: host arrays of nprob descriptors as for
 * crp_batch_create.  cache_path as for crp_autotune (key: device, sample
 * size, terms per problem, mode).  Creates and destroys batches;
 * synchronises. */
crp_status crp_autotune_batch(const crp_plan_desc *base, int32_t nprob, const crp_sparse *A,
                              const crp_sparse *B, int32_t sample_probs, const char *cache_path,
                              crp_plan_desc *best, double *best_terms_per_s, void *stream);

/* Library version string. */
const char *crp_version(void);

/* Message for the calling thread's last error ("" if none). */
const char *crp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* CRP_H */
