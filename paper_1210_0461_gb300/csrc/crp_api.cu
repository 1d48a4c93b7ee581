// Host side of the C ABI declared in include/crp.h: plan creation and
// validation, table sizing, launch configuration, status, top-k driver,
// export and statistics.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <unordered_map>
#include <vector>

#include "crp_internal.cuh"
#include "crp_topk.cuh"

using namespace crp;

namespace crp {
cudaError_t launch_export_range(const Slot *slots, const unsigned long long *part_off,
                                const unsigned long long *part_mask, uint32_t p0, uint32_t p1,
                                const unsigned long long *base, int value_type, int32_t *i_out,
                                int32_t *j_out, double *w_out, double *wl_out, cudaStream_t s);
}

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------

static thread_local std::string g_last_error;

static crp_status fail(crp_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

#define CRP_CUDA(call)                                                                         \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess)                                                                 \
            return fail(_e == cudaErrorMemoryAllocation ? CRP_ENOMEM : CRP_ECUDA,              \
                        std::string(#call) + ": " + cudaGetErrorString(_e));                   \
    } while (0)

extern "C" const char *crp_last_error(void) { return g_last_error.c_str(); }

namespace crp {
void set_last_error(const std::string &msg) { g_last_error = msg; }
}
extern "C" const char *crp_version(void) { return "crp 0.1.0 (sm_103a)"; }

// ---------------------------------------------------------------------------
// Hash parameters: SplitMix64 (Steele, Lea, Flood 2014) from each seed
// ---------------------------------------------------------------------------

static uint64_t splitmix64_next(uint64_t &state) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static SideHash make_side_hash(uint64_t seed, uint32_t logP) {
    SideHash h;
    uint64_t st = seed;
    h.a = splitmix64_next(st);
    h.b = splitmix64_next(st);
    h.shift = 64u - (logP > 0 ? logP : 1u);
    h.mask = (1u << logP) - 1u;
    return h;
}

// Count-Sketch signs: the third and fourth SplitMix64 outputs of each seed
static SignPair make_sign_pair(uint64_t seed_a, uint64_t seed_b) {
    SignPair s;
    uint64_t st = seed_a;
    splitmix64_next(st);
    splitmix64_next(st);
    s.ca = splitmix64_next(st);
    s.da = splitmix64_next(st);
    st = seed_b;
    splitmix64_next(st);
    splitmix64_next(st);
    s.cb = splitmix64_next(st);
    s.db = splitmix64_next(st);
    return s;
}

// ---------------------------------------------------------------------------
// Plan
// ---------------------------------------------------------------------------

struct crp_plan {
    crp_plan_desc d;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    HashPair hp;
    uint32_t logP = 0;
    // exact tables
    Slot *slots = nullptr;
    uint64_t n_slots = 0;
    std::vector<unsigned long long> h_off, h_mask;
    unsigned long long *d_off = nullptr, *d_mask = nullptr;
    unsigned int *d_full = nullptr;
    SpillRec *spill = nullptr;
    uint64_t spill_cap = 0;
    DevCounters *dc = nullptr;
    unsigned long long *d_scratch64 = nullptr;  // 2*P + 8 u64 of small scratch
    unsigned int *d_topk_hist = nullptr;
    // sorted-b scratch (G > 1)
    int32_t *s_idx = nullptr;
    float *s_val = nullptr;
    uint32_t *s_hash = nullptr;
    unsigned int *s_long = nullptr;
    uint64_t s_nnz_cap = 0, s_k_cap = 0;
    // launch configuration
    uint32_t G = 1, tile = 64, S = 8192;
    uint32_t q = 0, r = 0;  // owned partition interval [q, r)
    int grid = 0, grid_direct = 0;
    bool tables_ready = false;
    float summary_ms = 0.f;
    // summary mode
    bool summary = false;
    uint32_t ell = 0;
    unsigned int *d_live = nullptr, *d_floor = nullptr;
    Slot *d_ctmp = nullptr;
    int ctmp_grid = 0;
    SpillRec *d_spill2 = nullptr;
    unsigned long long res_off = 0, res_mask = 0;
    unsigned long long *d_res_keys = nullptr;
    unsigned int *d_res_bits = nullptr;  // row bits then column bits
    int32_t n_res = 0;
    // hot block (direct mode)
    uint32_t hot_R = 0;
    unsigned int *d_hot = nullptr, *d_cnt_a = nullptr, *d_cnt_b = nullptr, *d_sel = nullptr;
    uint16_t *d_rank_a = nullptr, *d_rank_b = nullptr;
    int64_t *d_items_a = nullptr, *d_items_b = nullptr;
    uint32_t warm_W = 0;
    // summary mode: the ragged block of reserved pairs (rows, cells per row,
    // first cell of each row, the reserved cells' indices)
    uint32_t resv_rows = 0;
    uint64_t resv_cells = 0;
    unsigned int *d_resv_len = nullptr, *d_resv_off = nullptr, *d_resv_idx = nullptr;
    unsigned int *d_warm_a = nullptr, *d_warm_b = nullptr;
    uint16_t *d_wrank_a = nullptr, *d_wrank_b = nullptr;
    int64_t *d_witems_a = nullptr, *d_witems_b = nullptr;
    // routed mode: pool of record chunks, their bins and the grouping by bin
    void *pool = nullptr;
    uint64_t pool_bytes = 0;
    uint32_t pool_chunks = 0, B = 0;
    unsigned int *d_chunk_bin = nullptr, *d_order = nullptr;
    // chunk counter, count[B], fill[B], start[B + 1], overflow counter
    unsigned int *d_route_ctl = nullptr;
    uint32_t ov_chunks = 0;             // overflow chunks at the start of the pool
    // P = 0 in the descriptor: a placeholder until the first call tunes the plan
    bool tune_first = false;
    crp_plan_desc user_desc = {};
    // certified top-k: cumulative degrees of rows and columns since the last
    // reset, the hot pairs' candidate buffer, calls answered from it
    unsigned long long *d_deg_a = nullptr, *d_deg_b = nullptr;
    bool warm_in_hot = false;      // warm items = the first warm_W hot items
    bool deg_b_mirrors_a = true;   // every call since the reset had B == A: d_deg_b unused
    TopkCand *d_hot_cand = nullptr;
    // top-k scratch kept across calls
    TopkCand *d_cand_keep = nullptr, *d_cand_sel = nullptr, *d_cand_tmp = nullptr;
    uint64_t cand_keep_cap = 0, cand_sel_cap = 0, cand_tmp_cap = 0;
    unsigned char *d_topk_stage = nullptr;
    uint64_t topk_stage_cap = 0;
    uint64_t topk_certified = 0;
    // locked-bucket summaries: a lock word per partition
    bool locked = false;
    unsigned int *d_locks = nullptr;
    // Count-Sketch: P estimators (int64 or fp64) and the sign hash
    void *d_sketch = nullptr;
    SignPair sg = {0, 0, 0, 0};
    // timing of the enumeration kernel and a count of our launches
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, evm = nullptr;
    // pinned words for counts read back mid-call, and the event that marks
    // their copy (the stream runs on while the host waits for it)
    unsigned long long *h_counts = nullptr;
    cudaEvent_t ev_counts = nullptr;
    bool timed = false, timed_mid = false;
    uint64_t launches = 0;
    // distinct entries of the whole product estimated from the sampled
    // partition group (0: the tables were not sized from a sample)
    uint64_t est_entries = 0;
};

static bool is_pow2(uint64_t x) { return x && !(x & (x - 1)); }
static uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

static crp_status alloc_tables(crp_plan *pl, uint64_t cap_per_partition) {
    const uint32_t P = pl->d.P;
    cap_per_partition = next_pow2(std::max<uint64_t>(cap_per_partition, 64));
    pl->h_off.resize(P);
    pl->h_mask.resize(P);
    // partitions outside the plan's interval get no slots (capacity 0: the
    // mask sentinel ~0 makes mask + 1 == 0)
    uint64_t total = 0;
    for (uint32_t p = 0; p < P; ++p) {
        const bool own = p >= pl->q && p < pl->r;
        pl->h_off[p] = total;
        pl->h_mask[p] = own ? cap_per_partition - 1 : ~0ull;
        if (own) total += cap_per_partition;
    }
    if (pl->slots) cudaFree(pl->slots);
    pl->slots = nullptr;
    CRP_CUDA(cudaMalloc(&pl->slots, total * sizeof(Slot)));
    pl->n_slots = total;
    CRP_CUDA(cudaMemcpyAsync(pl->d_off, pl->h_off.data(), P * sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_mask, pl->h_mask.data(), P * sizeof(unsigned long long),
                             cudaMemcpyHostToDevice, pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->d_full, 0, P * sizeof(unsigned int), pl->stream));
    CRP_CUDA(launch_fill_empty(pl->slots, total, pl->stream));
    pl->launches += 1;
    if (!pl->spill) {
        pl->spill_cap = std::max<uint64_t>(1u << 20, std::min<uint64_t>(total / 4, 1ull << 25));
        CRP_CUDA(cudaMalloc(&pl->spill, pl->spill_cap * sizeof(SpillRec)));
    }
    pl->tables_ready = true;
    return CRP_OK;
}

// Summary mode: every partition gets a table of next_pow2(4 ell) slots (at
// most 2 ell occupied between compactions), followed by the reserved-counter
// region; floors and live counts start at zero.
static crp_status alloc_summary(crp_plan *pl) {
    const uint32_t P = pl->d.P;
    pl->summary = true;
    pl->ell = pl->d.summary_counters;
    pl->locked = (pl->d.flags & CRP_PLAN_LOCKED_SUMMARY) != 0;
    // locked buckets: exactly ell counters used of next_pow2(ell) slots
    const uint64_t cap = pl->locked ? next_pow2(pl->ell)
                                    : next_pow2(std::max<uint64_t>(4ull * pl->ell, 64));
    const uint64_t rcap = pl->d.reserved_counters
                              ? next_pow2(std::max<uint64_t>(2ull * pl->d.reserved_counters, 64))
                              : 0;
    pl->h_off.resize(P);
    pl->h_mask.resize(P);
    for (uint32_t p = 0; p < P; ++p) {
        pl->h_off[p] = (unsigned long long)p * cap;
        pl->h_mask[p] = cap - 1;
    }
    const uint64_t total = (uint64_t)P * cap + rcap;
    CRP_CUDA(cudaMalloc(&pl->slots, total * sizeof(Slot)));
    pl->n_slots = total;
    pl->res_off = (uint64_t)P * cap;
    pl->res_mask = rcap ? rcap - 1 : 0;
    CRP_CUDA(cudaMemcpyAsync(pl->d_off, pl->h_off.data(), P * 8, cudaMemcpyHostToDevice,
                             pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_mask, pl->h_mask.data(), P * 8, cudaMemcpyHostToDevice,
                             pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->d_full, 0, P * 4, pl->stream));
    CRP_CUDA(cudaMalloc(&pl->d_live, P * 4));
    CRP_CUDA(cudaMalloc(&pl->d_floor, P * 4));
    CRP_CUDA(cudaMemsetAsync(pl->d_live, 0, P * 4, pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->d_floor, 0, P * 4, pl->stream));
    CRP_CUDA(launch_fill_empty(pl->slots, total, pl->stream));
    pl->launches += 1;
    pl->spill_cap = std::max<uint64_t>(1u << 20, std::min<uint64_t>((uint64_t)P * pl->ell, 1ull << 25));
    CRP_CUDA(cudaMalloc(&pl->spill, pl->spill_cap * sizeof(SpillRec)));
    CRP_CUDA(cudaMalloc(&pl->d_spill2, pl->spill_cap * sizeof(SpillRec)));
    pl->ctmp_grid = (int)std::min<uint32_t>(P, (uint32_t)pl->sm_count);
    CRP_CUDA(cudaMalloc(&pl->d_ctmp, (size_t)pl->ctmp_grid * pl->ell * sizeof(Slot)));
    if (pl->locked) {
        CRP_CUDA(cudaMalloc(&pl->d_locks, (size_t)P * 8));   // ticket, serving
        CRP_CUDA(cudaMemsetAsync(pl->d_locks, 0, (size_t)P * 8, pl->stream));
    }
    if (pl->d.reserved_counters) {
        CRP_CUDA(cudaMalloc(&pl->d_res_keys, (size_t)pl->d.reserved_counters * 8));
        const size_t words = (size_t)(pl->d.n_rows + 31) / 32 + (size_t)(pl->d.n_cols + 31) / 32;
        CRP_CUDA(cudaMalloc(&pl->d_res_bits, words * 4));
        CRP_CUDA(cudaMemsetAsync(pl->d_res_bits, 0, words * 4, pl->stream));
    }
    pl->tables_ready = true;
    return CRP_OK;
}

extern "C" crp_status crp_plan_create(crp_plan **out, const crp_plan_desc *desc, void *stream) {
    if (!out || !desc) return fail(CRP_EINVAL, "crp_plan_create: null argument");
    *out = nullptr;
    const crp_plan_desc &d = *desc;
    if (d.n_rows <= 0 || d.n_cols <= 0) return fail(CRP_EINVAL, "n_rows and n_cols must be > 0");
    if (d.P == 0) {   // tuned at the first call: a valid single-partition placeholder until then
        if (d.summary_counters || d.part_begin || d.part_end)
            return fail(CRP_EINVAL, "P = 0 (tuned at the first call) is for exact plans over all "
                                    "partitions");
        crp_plan_desc ph = d;
        ph.P = 1;
        ph.groups = 0;
        ph.hot_items = ph.warm_items = 0;
        ph.table_capacity_hint = 0;
        ph.flags &= ~(uint32_t)CRP_PLAN_ROUTED;
        crp_status st = crp_plan_create(out, &ph, stream);
        if (st != CRP_OK) return st;
        (*out)->tune_first = true;
        (*out)->user_desc = d;
        return CRP_OK;
    }
    if (!is_pow2(d.P) || d.P > (1u << 24))
        return fail(CRP_EINVAL, "P must be a power of two in [1, 2^24]");
    if (d.value_type != CRP_I32 && d.value_type != CRP_F32_COMP)
        return fail(CRP_EINVAL, "unknown value_type");
    if (d.mode != CRP_FULL && d.mode != CRP_UPPER) return fail(CRP_EINVAL, "unknown mode");
    if (d.target_load_pct > 90) return fail(CRP_EINVAL, "target_load_pct must be <= 90");
    if ((d.part_begin || d.part_end) &&
        (d.part_begin >= d.part_end || d.part_end > d.P || d.summary_counters))
        return fail(CRP_EINVAL, "partition interval must satisfy 0 <= begin < end <= P "
                                "(exact mode only)");
    if (d.smem_slots && (!is_pow2(d.smem_slots) || d.smem_slots < 4096 || d.smem_slots > 16384))
        return fail(CRP_EINVAL, "smem_slots must be a power of two in [4096, 16384]");
    if (d.groups && (!is_pow2(d.groups) || d.groups > d.P))
        return fail(CRP_EINVAL, "groups must be a power of two <= P");
    const bool locked = (d.flags & CRP_PLAN_LOCKED_SUMMARY) != 0;
    if (locked && (d.summary_counters < 1 || d.summary_counters > 64 || d.reserved_counters ||
                   (d.flags & CRP_PLAN_ROUTED)))
        return fail(CRP_EINVAL, "CRP_PLAN_LOCKED_SUMMARY needs 1 <= summary_counters <= 64, no "
                                "reserved_counters, not CRP_PLAN_ROUTED");
    if ((d.hot_items || d.warm_items) &&
        (d.hot_items > 4096 || d.warm_items > 4096 || d.value_type != CRP_I32 ||
         !(d.flags & (CRP_PLAN_DIRECT | CRP_PLAN_ROUTED)) || (d.summary_counters && !locked)))
        return fail(CRP_EINVAL, "hot_items / warm_items need CRP_PLAN_DIRECT or CRP_PLAN_ROUTED, "
                                "CRP_I32, <= 4096, and exact or locked-bucket tables");
    if (d.summary_counters && d.value_type != CRP_I32)
        return fail(CRP_EUNSUPPORTED, "summaries count {0,1} inputs (CRP_I32) only");
    if ((d.flags & CRP_PLAN_SKETCH) && (d.flags & CRP_PLAN_ROUTED))
        return fail(CRP_EINVAL, "CRP_PLAN_SKETCH is not available with CRP_PLAN_ROUTED");
    if (d.summary_counters > (1u << 24))
        return fail(CRP_EINVAL, "summary_counters must be <= 2^24 per partition");
    if (d.reserved_counters > (1u << 24))
        return fail(CRP_EINVAL, "reserved_counters must be <= 2^24");
    crp_plan *pl = new crp_plan();
    pl->d = d;
    pl->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&pl->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&pl->sm_count, cudaDevAttrMultiProcessorCount, pl->device);
    if (e != cudaSuccess) {
        delete pl;
        return fail(CRP_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    pl->logP = 0;
    while ((1u << pl->logP) < d.P) ++pl->logP;
    pl->hp.ha = make_side_hash(d.seed_a, pl->logP);
    pl->hp.hb = make_side_hash(d.seed_b, pl->logP);
    pl->G = d.groups ? d.groups : 1u;
    pl->q = (d.part_begin || d.part_end) ? d.part_begin : 0u;
    pl->r = (d.part_begin || d.part_end) ? d.part_end : d.P;
    pl->tile = d.tile_vectors ? d.tile_vectors : 64u;
    pl->S = d.smem_slots ? d.smem_slots : 8192u;
    crp_status st = CRP_OK;
#define ALLOC(ptr, bytes)                                                                      \
    if (st == CRP_OK && cudaMalloc(&(ptr), (bytes)) != cudaSuccess)                            \
        st = fail(CRP_ENOMEM, "device allocation failed");
    ALLOC(pl->d_off, d.P * sizeof(unsigned long long));
    ALLOC(pl->d_mask, d.P * sizeof(unsigned long long));
    ALLOC(pl->d_full, d.P * sizeof(unsigned int));
    ALLOC(pl->dc, sizeof(DevCounters));
    ALLOC(pl->d_scratch64, (2ull * d.P + 16) * sizeof(unsigned long long));
    ALLOC(pl->d_topk_hist, (kTopkBuckets + 512) * sizeof(unsigned int));
    if (d.flags & CRP_PLAN_SKETCH) {
        ALLOC(pl->d_sketch, (size_t)d.P * 8);
        if (st == CRP_OK && cudaMemsetAsync(pl->d_sketch, 0, (size_t)d.P * 8, pl->stream) !=
                                cudaSuccess)
            st = fail(CRP_ECUDA, "memset failed");
        pl->sg = make_sign_pair(d.seed_a, d.seed_b);
    }
#undef ALLOC
    if (st == CRP_OK && cudaMemsetAsync(pl->dc, 0, sizeof(DevCounters), pl->stream) != cudaSuccess)
        st = fail(CRP_ECUDA, "memset failed");
    if (st == CRP_OK) {
        int per_sm = accumulate_max_blocks_per_sm(d.value_type, pl->S,
                                                  (d.flags & CRP_PLAN_DIRECT) != 0);
        if (per_sm <= 0) st = fail(CRP_ECUDA, "accumulate kernel cannot be resident");
        pl->grid = per_sm * pl->sm_count;
        pl->grid_direct = accumulate_max_blocks_per_sm(d.value_type, pl->S, true) * pl->sm_count;
    }
    if (st == CRP_OK && (cudaEventCreate(&pl->ev0) != cudaSuccess ||
                         cudaEventCreate(&pl->ev1) != cudaSuccess ||
                         cudaEventCreate(&pl->evm) != cudaSuccess))
        st = fail(CRP_ECUDA, "cudaEventCreate failed");
    if (st == CRP_OK && d.summary_counters) {
        st = alloc_summary(pl);
    } else if (st == CRP_OK && d.table_capacity_hint) {
        uint64_t per = (d.table_capacity_hint + d.P - 1) / d.P;
        st = alloc_tables(pl, per);
    }
    if (st != CRP_OK) {
        crp_plan_destroy(pl);
        return st;
    }
    *out = pl;
    return CRP_OK;
}

extern "C" void crp_plan_destroy(crp_plan *pl) {
    if (!pl) return;
    cudaStreamSynchronize(pl->stream);
    cudaFree(pl->slots);
    cudaFree(pl->d_off);
    cudaFree(pl->d_mask);
    cudaFree(pl->d_full);
    cudaFree(pl->spill);
    cudaFree(pl->dc);
    cudaFree(pl->d_scratch64);
    cudaFree(pl->d_topk_hist);
    cudaFree(pl->s_idx);
    cudaFree(pl->s_val);
    cudaFree(pl->s_hash);
    cudaFree(pl->s_long);
    cudaFree(pl->d_hot);
    cudaFree(pl->d_cnt_a);
    cudaFree(pl->d_cnt_b);
    cudaFree(pl->d_sel);
    cudaFree(pl->d_rank_a);
    cudaFree(pl->d_rank_b);
    cudaFree(pl->d_items_a);
    cudaFree(pl->d_items_b);
    cudaFree(pl->d_resv_len);
    cudaFree(pl->d_resv_off);
    cudaFree(pl->d_resv_idx);
    cudaFree(pl->d_warm_a);
    cudaFree(pl->d_warm_b);
    cudaFree(pl->d_wrank_a);
    cudaFree(pl->d_wrank_b);
    cudaFree(pl->d_witems_a);
    cudaFree(pl->d_witems_b);
    cudaFree(pl->d_live);
    cudaFree(pl->d_floor);
    cudaFree(pl->d_ctmp);
    cudaFree(pl->d_spill2);
    cudaFree(pl->d_res_keys);
    cudaFree(pl->d_res_bits);
    cudaFree(pl->pool);
    cudaFree(pl->d_chunk_bin);
    cudaFree(pl->d_order);
    cudaFree(pl->d_route_ctl);
    cudaFree(pl->d_sketch);
    cudaFree(pl->d_locks);
    cudaFree(pl->d_deg_a);
    cudaFree(pl->d_deg_b);
    cudaFree(pl->d_hot_cand);
    cudaFree(pl->d_cand_keep);
    cudaFree(pl->d_cand_sel);
    cudaFree(pl->d_cand_tmp);
    cudaFree(pl->d_topk_stage);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    if (pl->evm) cudaEventDestroy(pl->evm);
    if (pl->ev_counts) cudaEventDestroy(pl->ev_counts);
    if (pl->h_counts) cudaFreeHost(pl->h_counts);
    delete pl;
}

extern "C" crp_status crp_reset(crp_plan *pl) {
    if (!pl) return fail(CRP_EINVAL, "null plan");
    CRP_CUDA(cudaMemsetAsync(pl->dc, 0, sizeof(DevCounters), pl->stream));
    if (pl->d_sketch) CRP_CUDA(cudaMemsetAsync(pl->d_sketch, 0, (size_t)pl->d.P * 8, pl->stream));
    if (pl->tables_ready) {
        CRP_CUDA(launch_fill_empty(pl->slots, pl->n_slots, pl->stream));
        pl->launches += 1;
        CRP_CUDA(cudaMemsetAsync(pl->d_full, 0, pl->d.P * sizeof(unsigned int), pl->stream));
    }
    if (pl->d_locks) CRP_CUDA(cudaMemsetAsync(pl->d_locks, 0, (size_t)pl->d.P * 8, pl->stream));
    if (pl->d_deg_a) {
        CRP_CUDA(cudaMemsetAsync(pl->d_deg_a, 0, (size_t)pl->d.n_rows * 8, pl->stream));
        CRP_CUDA(cudaMemsetAsync(pl->d_deg_b, 0, (size_t)pl->d.n_cols * 8, pl->stream));
    }
    pl->deg_b_mirrors_a = true;
    if (pl->summary) {
        CRP_CUDA(cudaMemsetAsync(pl->d_live, 0, pl->d.P * 4, pl->stream));
        CRP_CUDA(cudaMemsetAsync(pl->d_floor, 0, pl->d.P * 4, pl->stream));
        if (pl->n_res) {  // reserved keys stay registered; their counts restart at 0
            CRP_CUDA(launch_reserve_insert(pl->slots, pl->res_off, pl->res_mask, pl->d_res_keys,
                                           pl->n_res, pl->stream));
            pl->launches += 1;
        }
        if (pl->resv_rows)
            CRP_CUDA(launch_reserve_cells(pl->d_resv_idx, (int32_t)pl->n_res, pl->d_hot,
                                          pl->resv_cells, pl->stream));
    }
    return CRP_OK;
}

__global__ void k_take_ticket(unsigned int *next) { atomicAdd(next, 1u); }

extern "C" crp_status crp_debug_hold_lock(crp_plan *pl, uint32_t p) {
    if (!pl || !pl->locked || !pl->d_locks || p >= pl->d.P)
        return fail(CRP_EINVAL, "crp_debug_hold_lock: a locked-bucket plan and p < P are needed");
    k_take_ticket<<<1, 1, 0, pl->stream>>>(pl->d_locks + 2 * (size_t)p);
    CRP_CUDA(cudaGetLastError());
    pl->launches += 1;
    return CRP_OK;
}

extern "C" uint32_t crp_partition_of(const crp_plan *pl, int32_t i, int32_t j) {
    if (!pl) return 0;
    return partition_hash(pl->hp, (uint32_t)i, (uint32_t)j);
}

// ---------------------------------------------------------------------------
// Accumulate
// ---------------------------------------------------------------------------

static crp_status check_sparse(const crp_sparse *s, const char *name) {
    if (!s) return fail(CRP_EINVAL, std::string(name) + " is null");
    if (s->n_major < 0 || s->nnz < 0 || s->n_minor <= 0)
        return fail(CRP_EINVAL, std::string(name) + ": negative size");
    if (s->n_major > 0 && !s->ptr) return fail(CRP_EINVAL, std::string(name) + ": null ptr");
    if (s->nnz > 0 && !s->idx) return fail(CRP_EINVAL, std::string(name) + ": null idx");
    return CRP_OK;
}

static crp_status ensure_sort_scratch(crp_plan *pl, uint64_t nnz, uint64_t K, bool values) {
    if (nnz > pl->s_nnz_cap || (values && !pl->s_val && nnz)) {
        cudaFree(pl->s_idx);
        cudaFree(pl->s_val);
        cudaFree(pl->s_hash);
        pl->s_idx = nullptr;
        pl->s_val = nullptr;
        pl->s_hash = nullptr;
        uint64_t cap = std::max<uint64_t>(nnz, 1);
        CRP_CUDA(cudaMalloc(&pl->s_idx, cap * sizeof(int32_t)));
        CRP_CUDA(cudaMalloc(&pl->s_hash, cap * sizeof(uint32_t)));
        if (values) CRP_CUDA(cudaMalloc(&pl->s_val, cap * sizeof(float)));
        pl->s_nnz_cap = cap;
    }
    if (K > pl->s_k_cap) {
        cudaFree(pl->s_long);
        pl->s_long = nullptr;
        uint64_t cap = std::max<uint64_t>(K, 1);
        CRP_CUDA(cudaMalloc(&pl->s_long, cap * sizeof(unsigned int)));
        pl->s_k_cap = cap;
    }
    return CRP_OK;
}

static TableView table_view(crp_plan *pl, Slot *slots, const unsigned long long *off,
                            const unsigned long long *mask) {
    TableView tv;
    tv.slots = slots;
    tv.part_off = off;
    tv.part_mask = mask;
    tv.part_full = pl->d_full;
    tv.spill = pl->spill;
    tv.spill_cap = pl->spill_cap;
    tv.dc = pl->dc;
    tv.value_type = pl->d.value_type;
    tv.summary = pl->summary ? (pl->locked ? 2 : 1) : 0;
    tv.locks = pl->d_locks;
    if (pl->d.lock_wait_us) tv.lock_wait = (long long)pl->d.lock_wait_us * 2000;
    tv.bucket_ell = pl->ell;
    tv.live = pl->d_live;
    tv.floor = pl->d_floor;
    tv.hard_cap = 2u * pl->ell;
    tv.res_off = pl->res_off;
    tv.res_mask = pl->res_mask;
    tv.has_reserved = (pl->summary && pl->n_res > 0) ? 1 : 0;
    if (pl->d_res_bits) {
        tv.res_bits_a = pl->d_res_bits;
        tv.res_bits_b = pl->d_res_bits + (pl->d.n_rows + 31) / 32;
    }
    return tv;
}

// Shared-memory copies of the sketch in the direct kernel (decided once
// a.direct is final).
static void set_sketch_copies(const crp_plan *pl, AccumulateArgs &a) {
    a.sketch_smem = (a.sketch && a.direct && pl->d.P <= kSketchSmemMaxP)
                        ? std::min<uint32_t>(kSketchSmemMaxP / pl->d.P, 16u)
                        : 0u;
}

static AccumulateArgs make_args(crp_plan *pl, const crp_sparse *A, const crp_sparse *B,
                                const int32_t *b_idx, const float *b_val, uint32_t G) {
    AccumulateArgs a;
    a.a_ptr = A->ptr;
    a.a_idx = A->idx;
    a.a_val = A->val;
    a.b_ptr = B->ptr;
    a.b_idx = b_idx;
    a.b_val = b_val;
    a.K = A->n_major;
    a.n_rows = pl->d.n_rows;
    a.n_cols = pl->d.n_cols;
    a.groups = G;
    a.group_begin = 0;
    a.group_end = G;
    a.tile = pl->tile;
    a.n_tiles = (uint32_t)((A->n_major + pl->tile - 1) / pl->tile);
    a.mode = pl->d.mode;
    a.use_match = (pl->d.flags & CRP_PLAN_NO_WARP_MATCH) ? 0 : 1;
    a.debug_checks = (pl->d.flags & CRP_PLAN_DEBUG_CHECKS) ? 1 : 0;
    a.direct = (pl->d.flags & CRP_PLAN_DIRECT) ? 1 : 0;
    // T^T T above the diagonal with A and B the same sorted lists: enumerate
    // only j after i (rows must hold distinct ascending indices)
    a.sym_upper = (pl->d.mode == CRP_UPPER && G == 1 && A->ptr == B->ptr && A->idx == B->idx &&
                   b_idx == B->idx && (pl->d.flags & CRP_PLAN_SORTED_ROWS)) ? 1 : 0;
    if (pl->q != 0 || pl->r != pl->d.P) {
        const uint32_t w = pl->d.P / G;
        if (G > 1 && pl->q % w == 0 && pl->r % w == 0) {
            a.group_begin = pl->q / w;   // Lemma 1: enumerate only the owned groups
            a.group_end = pl->r / w;
        } else {
            a.part_lo = pl->q;           // otherwise keep only the owned terms
            a.part_hi = pl->r;
        }
    }
    a.smem_slots = pl->S;
    a.hp = pl->hp;
    if (pl->d_sketch) {
        a.sketch = pl->d_sketch;
        a.sg = pl->sg;
    }
    set_sketch_copies(pl, a);
    return a;
}

// Estimate the number of distinct entries (nonzeros of A B) from one group of
// partitions: the terms hashing into partitions [0, P/Gs) are accumulated
// exactly into a scratch table (Lemma 1 keeps that pass linear in the input
// plus those terms), and their distinct count is scaled by Gs.  h is pairwise
// independent, so each group holds ~1/Gs of the entries.  This is how the
// paper's remark on estimating nnz(AB) from a sample of the output (Section 4,
// "Parameters") is realised with the partition structure itself.
static crp_status estimate_and_allocate(crp_plan *pl, const crp_sparse *A, const crp_sparse *B,
                                        const int32_t *b_idx, const float *b_val) {
    const uint32_t P = pl->d.P;
    CRP_CUDA(launch_count_terms(A->ptr, B->ptr, A->n_major, pl->d_scratch64, pl->stream));
    unsigned long long terms = 0;
    CRP_CUDA(cudaMemcpyAsync(&terms, pl->d_scratch64, 8, cudaMemcpyDeviceToHost, pl->stream));
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    const uint64_t bound = std::min<uint64_t>(terms, (uint64_t)pl->d.n_rows * pl->d.n_cols);
    uint64_t distinct;
    const uint32_t Gs = std::min<uint32_t>(P, 64u);
    if (Gs <= 1 || bound < (1ull << 22)) {
        distinct = bound;
    } else {
        // scratch table for partitions [0, P/Gs) (others unused)
        const uint32_t np = P / Gs;
        const uint64_t cap = next_pow2(std::max<uint64_t>(2 * (bound / P + 1), 1024));
        Slot *tmp = nullptr;
        CRP_CUDA(cudaMalloc(&tmp, (uint64_t)np * cap * sizeof(Slot)));
        std::vector<unsigned long long> off(P, 0), mask(P, cap - 1);
        for (uint32_t p = 0; p < np; ++p) off[p] = (unsigned long long)p * cap;
        unsigned long long *d_off = pl->d_scratch64, *d_mask = pl->d_scratch64 + P;
        CRP_CUDA(cudaMemcpyAsync(d_off, off.data(), P * 8, cudaMemcpyHostToDevice, pl->stream));
        CRP_CUDA(cudaMemcpyAsync(d_mask, mask.data(), P * 8, cudaMemcpyHostToDevice, pl->stream));
        CRP_CUDA(launch_fill_empty(tmp, (uint64_t)np * cap, pl->stream));
        CRP_CUDA(cudaMemsetAsync(pl->d_full, 0, P * sizeof(unsigned int), pl->stream));
        CRP_CUDA(cudaMemsetAsync(pl->dc, 0, sizeof(DevCounters), pl->stream));
        // sorted b is needed for a group run
        const int32_t *sb_idx = b_idx;
        const float *sb_val = b_val;
        if (b_idx == B->idx) {
            crp_status st = ensure_sort_scratch(pl, B->nnz, B->n_major, B->val != nullptr);
            if (st != CRP_OK) { cudaFree(tmp); return st; }
            CRP_CUDA(launch_sort_by_hash(B->ptr, B->idx, B->val, B->n_major, pl->hp.hb, pl->s_idx,
                                         pl->s_val, pl->s_hash, pl->dc, pl->s_long, pl->sm_count,
                                         pl->stream));
            sb_idx = pl->s_idx;
            sb_val = B->val ? pl->s_val : nullptr;
        }
        AccumulateArgs a = make_args(pl, A, B, sb_idx, sb_val, Gs);
        a.sketch = nullptr;   // a sizing pass: the sketch counts the real pass only
        a.sketch_smem = 0;
        a.group_begin = 0;   // the sample is group 0 of the whole hash space,
        a.group_end = 1;     // whatever interval the plan owns
        a.part_lo = 0;
        a.part_hi = 0xFFFFFFFFu;
        a.hot_R = 0;
        a.warm_W = 0;
        a.tv = table_view(pl, tmp, d_off, d_mask);
        CRP_CUDA(launch_accumulate(a, pl->s_hash, pl->grid, pl->stream));
        // live entries per sampled partition
        std::vector<unsigned long long> live(np, 0);
        unsigned long long *d_live = nullptr, *d_terms = nullptr;
        CRP_CUDA(cudaMalloc(&d_live, np * 8));
        CRP_CUDA(cudaMalloc(&d_terms, np * 8));
        CRP_CUDA(launch_partition_sums(tmp, d_off, d_mask, np, pl->d.value_type, d_terms, d_live,
                                       pl->stream));
        CRP_CUDA(cudaMemcpyAsync(live.data(), d_live, np * 8, cudaMemcpyDeviceToHost, pl->stream));
        unsigned int status = 0;
        CRP_CUDA(cudaMemcpyAsync(&status, &pl->dc->status, 4, cudaMemcpyDeviceToHost, pl->stream));
        CRP_CUDA(cudaStreamSynchronize(pl->stream));
        cudaFree(d_live);
        cudaFree(d_terms);
        cudaFree(tmp);
        CRP_CUDA(cudaMemsetAsync(pl->dc, 0, sizeof(DevCounters), pl->stream));
        CRP_CUDA(cudaMemsetAsync(pl->d_full, 0, P * sizeof(unsigned int), pl->stream));
        if (status & (kStatusTableFull | kStatusSpillFull)) {
            distinct = bound;  // sample overflowed its bound: fall back
        } else {
            unsigned long long mx = 0, sum = 0;
            for (auto v : live) { mx = std::max(mx, v); sum += v; }
            distinct = std::max<uint64_t>((uint64_t)mx * P, (uint64_t)sum * Gs);
            pl->est_entries = (uint64_t)sum * Gs;
        }
    }
    // target load per partition (default 65%: capacities are powers of two, so
    // the tables hold between a third and two thirds of their slots)
    const double load = pl->d.target_load_pct ? pl->d.target_load_pct / 100.0 : 0.65;
    uint64_t per = (uint64_t)((double)distinct / P / load) + 64;
    return alloc_tables(pl, per);
}

static crp_status select_hot_items(crp_plan *pl, const crp_sparse *A, const crp_sparse *B);
static crp_status count_degrees(crp_plan *pl, const crp_sparse *A, const crp_sparse *B);
static void set_dense_args(crp_plan *pl, AccumulateArgs &a);
static crp_status flush_dense(crp_plan *pl, const TableView &tv);

// Compact every partition holding more than ell keys, then re-insert spilled
// updates (each re-insert may spill again when a partition refills; repeat).
static crp_status summary_settle(crp_plan *pl, bool final) {
    const uint32_t P = pl->d.P;
    const uint32_t trigger = final ? pl->ell : pl->ell + (3u * pl->ell) / 4u;
    for (int round = 0; round < 256; ++round) {
        CRP_CUDA(launch_summary_compact(pl->slots, pl->d_off, pl->d_mask, pl->d_live, pl->d_floor,
                                        nullptr, P, pl->ell, round == 0 ? trigger : pl->ell,
                                        pl->d_ctmp, pl->ctmp_grid, pl->stream));
        pl->launches += 1;
        unsigned long long n_spill = 0;
        CRP_CUDA(cudaMemcpyAsync(&n_spill, &pl->dc->spill_n, 8, cudaMemcpyDeviceToHost, pl->stream));
        CRP_CUDA(cudaStreamSynchronize(pl->stream));
        if (n_spill == 0) return CRP_OK;
        if (n_spill > pl->spill_cap)
            return fail(CRP_ETABLE_FULL, "summary spill list overflowed; counts were lost");
        CRP_CUDA(cudaMemcpyAsync(pl->d_spill2, pl->spill, n_spill * sizeof(SpillRec),
                                 cudaMemcpyDeviceToDevice, pl->stream));
        CRP_CUDA(cudaMemsetAsync(&pl->dc->spill_n, 0, 8, pl->stream));
        TableView tv = table_view(pl, pl->slots, pl->d_off, pl->d_mask);
        CRP_CUDA(launch_spill_reinsert(pl->d_spill2, n_spill, pl->hp, tv, pl->stream));
        pl->launches += 1;
    }
    return fail(CRP_ETABLE_FULL, "summary did not settle");
}

// Summary mode: the outer products are processed in chunks of about P * ell
// terms (about ell new keys per partition), each followed by compaction.
static crp_status summary_accumulate(crp_plan *pl, const crp_sparse *A, const crp_sparse *B) {
    const uint32_t P = pl->d.P;
    CRP_CUDA(launch_count_terms(A->ptr, B->ptr, A->n_major, pl->d_scratch64, pl->stream));
    unsigned long long terms = 0;
    CRP_CUDA(cudaMemcpyAsync(&terms, pl->d_scratch64, 8, cudaMemcpyDeviceToHost, pl->stream));
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    pl->launches += 1;
    // about ell / 4 new keys per partition per chunk at most, within the
    // headroom between the compaction trigger (7/4 ell) and the cap (2 ell)
    const uint64_t chunk_terms = std::max<uint64_t>((uint64_t)P * pl->ell / 4, 1);
    const uint64_t n_chunks = std::max<uint64_t>((terms + chunk_terms - 1) / chunk_terms, 1);
    const int64_t K = A->n_major;
    const int64_t kstep = (K + (int64_t)n_chunks - 1) / (int64_t)n_chunks;
    float total_ms = 0.f;
    for (int64_t k0 = 0; k0 < K; k0 += kstep) {
        const int64_t k1 = std::min(K, k0 + kstep);
        crp_sparse As = *A, Bs = *B;
        As.ptr = A->ptr + k0;
        As.n_major = k1 - k0;
        Bs.ptr = B->ptr + k0;
        Bs.n_major = k1 - k0;
        AccumulateArgs a = make_args(pl, &As, &Bs, B->idx, B->val, 1);
        a.direct = 1;
        set_sketch_copies(pl, a);
        a.tv = table_view(pl, pl->slots, pl->d_off, pl->d_mask);
        if (pl->resv_rows) {
            // the reserved pairs all fall in the ragged block: no reserved-key
            // test on the way to the summaries
            a.hot_rank_a = pl->d_rank_a;
            a.hot_rank_b = pl->d_rank_b;
            a.hot_block = pl->d_hot;
            a.hot_R = pl->resv_rows;
            a.resv_len = pl->d_resv_len;
            a.resv_off = pl->d_resv_off;
            a.tv.has_reserved = 0;
        }
        CRP_CUDA(cudaMemsetAsync(&pl->dc->work_next, 0, sizeof(unsigned int), pl->stream));
        CRP_CUDA(cudaEventRecord(pl->ev0, pl->stream));
        CRP_CUDA(launch_accumulate(a, nullptr, pl->grid_direct, pl->stream));
        if (pl->resv_rows && k1 == K) {
            CRP_CUDA(launch_reserve_flush(pl->d_hot, pl->resv_cells, pl->d_resv_off,
                                          pl->resv_rows, pl->d_items_a, pl->d_items_b, pl->hp,
                                          table_view(pl, pl->slots, pl->d_off, pl->d_mask),
                                          &pl->dc->flushed, pl->stream));
            pl->launches += 1;
        }
        CRP_CUDA(cudaEventRecord(pl->ev1, pl->stream));
        pl->launches += 1;
        crp_status st = summary_settle(pl, k1 == K);
        if (st != CRP_OK) return st;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pl->ev0, pl->ev1) == cudaSuccess) total_ms += ms;
    }
    pl->summary_ms = total_ms;
    pl->timed = false;
    return CRP_OK;
}

// The plan's pinned words and their event, made at first use.
static crp_status ensure_pinned(crp_plan *pl) {
    if (!pl->h_counts) {
        CRP_CUDA(cudaMallocHost(&pl->h_counts, 4 * sizeof(unsigned long long)));
        CRP_CUDA(cudaEventCreateWithFlags(&pl->ev_counts, cudaEventDisableTiming));
    }
    return CRP_OK;
}

// Routed mode: enumerate every term once into per-group bins, then apply the
// bins group by group so each group's table region stays in L2.
// Size the record pool and bins of the routed path for `records` records
// and fill RA's routing fields (RA.acc is the caller's).
static crp_status routed_prepare(crp_plan *pl, uint64_t records, RouteArgs &RA) {
    const uint32_t P = pl->d.P;
    // groups of partitions whose table region is about 96 MB or more (the
    // record chunks of every CTA stay open in L2 for each group, so more
    // groups cost the enumeration more than they save the apply phase), but
    // at least 256 groups: a CTA's appends to one group share one
    // shared-memory word, and fewer groups make those atomics contend
    const uint64_t table_bytes = pl->n_slots * sizeof(Slot);
    const uint64_t want = std::max<uint64_t>(table_bytes / (96ull << 20), 256);
    uint32_t Bn = 1;
    while (2ull * Bn <= want && Bn < P) Bn <<= 1;
    if (pl->d.groups) Bn = pl->G;  // explicit partition groups = bins
    Bn = std::min<uint32_t>(Bn, 8192);   // per-CTA chunk state lives in shared memory
    const int grid = 2 * pl->sm_count;
    const uint64_t rec = pl->d.value_type == CRP_I32 ? 8 : 16;
    // every record, 1/64 more for spares reserved ahead but never installed;
    // each CTA also holds a partly filled chunk and a spare per bin; overflow
    // chunks for appends that find no chunk slot: 1/256 of the chunks, at
    // least 256 (a pool that still runs dry sends records to the overflow
    // chunks, then straight to the tables)
    const uint32_t ovc = (uint32_t)std::min<uint64_t>(
        std::max<uint64_t>(records / kChunkRecs / 256, 256), 1u << 20);
    const uint64_t chunks_needed = (records + records / 64 + kChunkRecs - 1) / kChunkRecs +
                                   2ull * Bn * grid + ovc + 1;
    uint32_t chunks = (uint32_t)std::min<uint64_t>(chunks_needed, 0xFFFFFFF0ull);
    if (pl->d.route_pool_chunks)   // a capped pool (the overflow paths take the rest)
        chunks = std::min<uint32_t>(chunks, std::max<uint32_t>(pl->d.route_pool_chunks, ovc + 1));
    if (Bn != pl->B) {
        cudaFree(pl->d_route_ctl);
        pl->d_route_ctl = nullptr;
        pl->B = 0;
        CRP_CUDA(cudaMalloc(&pl->d_route_ctl, (3 * (size_t)Bn + 3) * 4));
        pl->B = Bn;
    }
    if (chunks > pl->pool_chunks) {
        cudaFree(pl->pool);
        cudaFree(pl->d_chunk_bin);
        cudaFree(pl->d_order);
        pl->pool = nullptr;
        pl->d_chunk_bin = pl->d_order = nullptr;
        pl->pool_chunks = 0;
        pl->pool_bytes = 0;
        // a smaller pool only sends the overflow straight to the tables
        uint32_t c = chunks;
        while (true) {
            if (cudaMalloc(&pl->pool, (size_t)c * kChunkRecs * rec) == cudaSuccess) break;
            cudaGetLastError();
            pl->pool = nullptr;
            if (c <= chunks / 16 || c <= ovc + 1) return fail(CRP_ENOMEM, "routed pool");
            c /= 2;
        }
        CRP_CUDA(cudaMalloc(&pl->d_chunk_bin, (size_t)c * 4));
        CRP_CUDA(cudaMalloc(&pl->d_order, (size_t)c * 4));
        pl->pool_chunks = c;
        pl->pool_bytes = (uint64_t)c * kChunkRecs * rec;
    }
    // chunks [0, ovc): overflow, bin 0, empty; the pool hands out chunks from ovc
    pl->ov_chunks = ovc;
    const uint32_t n_chunks = std::min<uint32_t>(pl->pool_chunks, chunks);
    CRP_CUDA(cudaMemsetAsync(pl->d_chunk_bin, 0xFF, (size_t)n_chunks * 4, pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->d_chunk_bin, 0, (size_t)ovc * 4, pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->pool, 0xFF, (size_t)ovc * kChunkRecs * rec, pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->d_route_ctl, 0, (2 * (size_t)Bn + 1) * 4, pl->stream));
    CRP_CUDA(cudaMemsetAsync(pl->d_route_ctl + 3 * (size_t)Bn + 2, 0, 4, pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_route_ctl, &pl->ov_chunks, 4, cudaMemcpyHostToDevice,
                             pl->stream));
    unsigned int *ctl = pl->d_route_ctl;
    RA.pool = pl->pool;
    RA.chunk_bin = pl->d_chunk_bin;
    RA.chunk_next = ctl;
    RA.order = pl->d_order;
    RA.start = ctl + 1 + 2 * Bn;
    RA.n_chunks = n_chunks;
    RA.B = Bn;
    uint32_t lgB = 0;
    while ((1u << lgB) < Bn) ++lgB;
    RA.B_shift = pl->logP - lgB;
    RA.core_H = std::min<uint32_t>(RA.acc.hot_R, 128);
    RA.ov_next = ctl + 3 * Bn + 2;
    RA.ov_cap = ovc * kChunkRecs;
    return CRP_OK;
}

// The two routed phases on the plan's stream (evm between them).
static crp_status routed_run(crp_plan *pl, const RouteArgs &RA) {
    CRP_CUDA(cudaMemsetAsync(&pl->dc->work_next, 0, sizeof(unsigned int), pl->stream));
    CRP_CUDA(launch_route(RA, pl->sm_count, pl->stream));
    CRP_CUDA(cudaEventRecord(pl->evm, pl->stream));
    CRP_CUDA(launch_apply(RA, pl->d_route_ctl + 1, pl->d_route_ctl + 1 + RA.B,
                          2 * pl->sm_count, pl->stream));
    pl->launches += 5;
    return CRP_OK;
}

// Routed mode: enumerate every term once into per-group bins, then apply the
// bins group by group so each group's table region stays in L2.
static crp_status routed_accumulate(crp_plan *pl, const crp_sparse *A, const crp_sparse *B) {
    crp_status st;
    RouteArgs RA;
    RA.acc = make_args(pl, A, B, B->idx, B->val, 1);
    RA.acc.tv = table_view(pl, pl->slots, pl->d_off, pl->d_mask);
    if (pl->d.hot_items || pl->d.warm_items) {
        st = select_hot_items(pl, A, B);
        if (st != CRP_OK) return st;
        set_dense_args(pl, RA.acc);
    }
    // the records this call routes (the terms outside the dense tiers) size
    // the pool: counted exactly on the first outer products (the sample the
    // tiers were chosen from), their routed share of the terms scaled to all
    // terms with a 10 % margin (a pool that still runs dry sends records to
    // the overflow chunks, then straight to the tables)
    const int64_t K = A->n_major;
    const int64_t S = std::min<int64_t>(K, std::max<int64_t>(65536, K / 64));
    AccumulateArgs sample = RA.acc;
    sample.K = S;
    // (the counts come back through pinned words while the stream goes on
    // to count the degrees for the top-k bound)
    st = ensure_pinned(pl);
    if (st != CRP_OK) return st;
    CRP_CUDA(launch_count_records(sample, pl->d_scratch64, pl->stream));
    CRP_CUDA(launch_count_terms(A->ptr, B->ptr, S, pl->d_scratch64 + 1, pl->stream));
    CRP_CUDA(launch_count_terms(A->ptr, B->ptr, K, pl->d_scratch64 + 2, pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->h_counts, pl->d_scratch64, 24, cudaMemcpyDeviceToHost,
                             pl->stream));
    CRP_CUDA(cudaEventRecord(pl->ev_counts, pl->stream));
    pl->launches += 3;
    if (pl->d.hot_items || pl->d.warm_items) {
        st = count_degrees(pl, A, B);
        if (st != CRP_OK) return st;
    }
    CRP_CUDA(cudaEventSynchronize(pl->ev_counts));
    // sample records, sample terms, all terms
    const unsigned long long cnt[3] = {pl->h_counts[0], pl->h_counts[1], pl->h_counts[2]};
    const double share = cnt[1] ? (double)cnt[0] / (double)cnt[1] : 1.0;
    const uint64_t records =
        std::min<uint64_t>(cnt[2], (uint64_t)(share * 1.1 * (double)cnt[2]) + 65536);
    st = routed_prepare(pl, records, RA);
    if (st != CRP_OK) return st;
    CRP_CUDA(cudaEventRecord(pl->ev0, pl->stream));
    st = routed_run(pl, RA);
    if (st != CRP_OK) return st;
    st = flush_dense(pl, RA.acc.tv);
    if (st != CRP_OK) return st;
    CRP_CUDA(cudaEventRecord(pl->ev1, pl->stream));
    pl->timed = true;
    pl->timed_mid = true;
    return CRP_OK;
}

// Dense tiers of this call: the R (hot) and W (warm) most frequent row
// indices of A and column indices of B over the first 1/64 of the outer
// products (at least 4096); ranks map an item to its row / column of the hot
// block or of a warm stripe.
static crp_status select_hot_items(crp_plan *pl, const crp_sparse *A, const crp_sparse *B) {
    const uint32_t nmin = (uint32_t)std::min(pl->d.n_rows, pl->d.n_cols);
    const uint32_t R = std::min<uint32_t>(pl->d.hot_items, nmin);
    uint32_t W = std::min<uint32_t>(pl->d.warm_items, nmin);
    const uint64_t stripe_cols = (uint64_t)pl->d.n_rows + pl->d.n_cols;
    while (W && (uint64_t)W * stripe_cols * 4 > (64ull << 20)) W >>= 1;
    cudaStream_t s = pl->stream;
    if (!pl->d_cnt_a) {
        CRP_CUDA(cudaMalloc(&pl->d_cnt_a, (size_t)pl->d.n_rows * 4));
        CRP_CUDA(cudaMalloc(&pl->d_cnt_b, (size_t)pl->d.n_cols * 4));
        CRP_CUDA(cudaMalloc(&pl->d_sel, 260 * 4));
        if (R) {
            CRP_CUDA(cudaMalloc(&pl->d_hot, (size_t)R * R * 4));
            CRP_CUDA(cudaMemsetAsync(pl->d_hot, 0, (size_t)R * R * 4, s));
            CRP_CUDA(cudaMalloc(&pl->d_rank_a, (size_t)pl->d.n_rows * 2));
            CRP_CUDA(cudaMalloc(&pl->d_rank_b, (size_t)pl->d.n_cols * 2));
            CRP_CUDA(cudaMalloc(&pl->d_items_a, (size_t)R * 8));
            CRP_CUDA(cudaMalloc(&pl->d_items_b, (size_t)R * 8));
        }
        if (W) {
            CRP_CUDA(cudaMalloc(&pl->d_warm_a, (size_t)W * pl->d.n_cols * 4));
            CRP_CUDA(cudaMalloc(&pl->d_warm_b, (size_t)W * pl->d.n_rows * 4));
            CRP_CUDA(cudaMemsetAsync(pl->d_warm_a, 0, (size_t)W * pl->d.n_cols * 4, s));
            CRP_CUDA(cudaMemsetAsync(pl->d_warm_b, 0, (size_t)W * pl->d.n_rows * 4, s));
            CRP_CUDA(cudaMalloc(&pl->d_wrank_a, (size_t)pl->d.n_rows * 2));
            CRP_CUDA(cudaMalloc(&pl->d_wrank_b, (size_t)pl->d.n_cols * 2));
            CRP_CUDA(cudaMalloc(&pl->d_witems_a, (size_t)W * 8));
            CRP_CUDA(cudaMalloc(&pl->d_witems_b, (size_t)W * 8));
        }
        pl->hot_R = R;
        pl->warm_W = W;
    }
    const int64_t K = A->n_major;
    const int64_t S = std::min<int64_t>(K, std::max<int64_t>(4096, K / 64));
    // the sample's nonzeros end at ptr[S], read by the counting kernel itself
    const int64_t hint_a = K ? (int64_t)((double)A->nnz * (double)S / (double)K) : 0;
    const int64_t hint_b = K ? (int64_t)((double)B->nnz * (double)S / (double)K) : 0;
    // A and B the same arrays (T^T T): one count and one selection serve
    // both sides, the B side a copy of the A side's items and ranks
    const bool mirror = A->idx == B->idx && A->ptr == B->ptr && pl->d.n_rows == pl->d.n_cols;
    CRP_CUDA(cudaMemsetAsync(pl->d_cnt_a, 0, (size_t)pl->d.n_rows * 4, s));
    if (!mirror) CRP_CUDA(cudaMemsetAsync(pl->d_cnt_b, 0, (size_t)pl->d.n_cols * 4, s));
    CRP_CUDA(launch_item_counts_at(A->idx, A->ptr + S, hint_a, pl->d.n_rows, pl->d_cnt_a, s));
    if (!mirror)
        CRP_CUDA(launch_item_counts_at(B->idx, B->ptr + S, hint_b, pl->d.n_cols, pl->d_cnt_b, s));
    pl->launches += mirror ? 1 : 2;
    if (pl->hot_R) {
        CRP_CUDA(select_top(pl->d_cnt_a, pl->d.n_rows, pl->hot_R, pl->d_items_a, pl->d_sel, s));
        // ranks in order of frequency: the lowest ranks are the heaviest items
        CRP_CUDA(order_by_count(pl->d_items_a, pl->d_cnt_a, pl->hot_R, s));
        CRP_CUDA(launch_hot_ranks(pl->d_rank_a, pl->d.n_rows, pl->d_items_a, pl->hot_R, s));
        if (mirror) {
            CRP_CUDA(cudaMemcpyAsync(pl->d_items_b, pl->d_items_a, (size_t)pl->hot_R * 8,
                                     cudaMemcpyDeviceToDevice, s));
            CRP_CUDA(cudaMemcpyAsync(pl->d_rank_b, pl->d_rank_a, (size_t)pl->d.n_cols * 2,
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            CRP_CUDA(select_top(pl->d_cnt_b, pl->d.n_cols, pl->hot_R, pl->d_items_b, pl->d_sel, s));
            CRP_CUDA(order_by_count(pl->d_items_b, pl->d_cnt_b, pl->hot_R, s));
            CRP_CUDA(launch_hot_ranks(pl->d_rank_b, pl->d.n_cols, pl->d_items_b, pl->hot_R, s));
        }
        pl->launches += mirror ? kSelectTopLaunches + 3 : 2 * kSelectTopLaunches + 6;
    }
    pl->warm_in_hot = pl->warm_W && pl->hot_R >= pl->warm_W;
    if (pl->warm_in_hot) {
        // the warm items are the first warm_W hot items (those are ordered by
        // count), so an item's warm rank is its hot rank: one class order of
        // the ranks serves both tiers in the routed walk
        const size_t wb = (size_t)pl->warm_W * 8;
        CRP_CUDA(cudaMemcpyAsync(pl->d_witems_a, pl->d_items_a, wb, cudaMemcpyDeviceToDevice, s));
        CRP_CUDA(launch_hot_ranks(pl->d_wrank_a, pl->d.n_rows, pl->d_witems_a, pl->warm_W, s));
        if (mirror) {
            CRP_CUDA(cudaMemcpyAsync(pl->d_witems_b, pl->d_witems_a, wb, cudaMemcpyDeviceToDevice,
                                     s));
            CRP_CUDA(cudaMemcpyAsync(pl->d_wrank_b, pl->d_wrank_a, (size_t)pl->d.n_cols * 2,
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            CRP_CUDA(cudaMemcpyAsync(pl->d_witems_b, pl->d_items_b, wb, cudaMemcpyDeviceToDevice,
                                     s));
            CRP_CUDA(launch_hot_ranks(pl->d_wrank_b, pl->d.n_cols, pl->d_witems_b, pl->warm_W, s));
        }
        pl->launches += mirror ? 2 : 4;
    } else if (pl->warm_W) {
        CRP_CUDA(select_top(pl->d_cnt_a, pl->d.n_rows, pl->warm_W, pl->d_witems_a, pl->d_sel, s));
        CRP_CUDA(launch_hot_ranks(pl->d_wrank_a, pl->d.n_rows, pl->d_witems_a, pl->warm_W, s));
        if (mirror) {
            CRP_CUDA(cudaMemcpyAsync(pl->d_witems_b, pl->d_witems_a, (size_t)pl->warm_W * 8,
                                     cudaMemcpyDeviceToDevice, s));
            CRP_CUDA(cudaMemcpyAsync(pl->d_wrank_b, pl->d_wrank_a, (size_t)pl->d.n_cols * 2,
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            CRP_CUDA(select_top(pl->d_cnt_b, pl->d.n_cols, pl->warm_W, pl->d_witems_b, pl->d_sel,
                                s));
            CRP_CUDA(launch_hot_ranks(pl->d_wrank_b, pl->d.n_cols, pl->d_witems_b, pl->warm_W, s));
        }
        pl->launches += mirror ? kSelectTopLaunches + 2 : 2 * kSelectTopLaunches + 4;
    }
    return CRP_OK;
}

// Degrees of every row and column over all calls since the reset (exact
// integer tables with a hot set): the bound that lets crp_topk answer from
// the hot pairs. Runs after select_hot_items (it reads the hot ranks).
static crp_status count_degrees(crp_plan *pl, const crp_sparse *A, const crp_sparse *B) {
    if (!pl->hot_R || pl->summary || pl->d.value_type != CRP_I32) return CRP_OK;
    cudaStream_t s = pl->stream;
    if (!pl->d_deg_a) {
        CRP_CUDA(cudaMalloc(&pl->d_deg_a, (size_t)pl->d.n_rows * 8));
        CRP_CUDA(cudaMalloc(&pl->d_deg_b, (size_t)pl->d.n_cols * 8));
        CRP_CUDA(cudaMemsetAsync(pl->d_deg_a, 0, (size_t)pl->d.n_rows * 8, s));
        CRP_CUDA(cudaMemsetAsync(pl->d_deg_b, 0, (size_t)pl->d.n_cols * 8, s));
    }
    // (B the same arrays as A, as for T^T T: one count serves both sides for
    // as long as every call since the reset is like that)
    const bool same = A->idx == B->idx && A->nnz == B->nnz && pl->d.n_rows == pl->d.n_cols;
    if (!same && pl->deg_b_mirrors_a) {
        CRP_CUDA(cudaMemcpyAsync(pl->d_deg_b, pl->d_deg_a, (size_t)pl->d.n_cols * 8,
                                 cudaMemcpyDeviceToDevice, s));
        pl->deg_b_mirrors_a = false;
    }
    CRP_CUDA(launch_degrees(A->idx, A->nnz, pl->d.n_rows, pl->d_rank_a, pl->hot_R, pl->d_items_a,
                            pl->d_deg_a, pl->sm_count, s));
    pl->launches += 1;
    if (!pl->deg_b_mirrors_a) {
        CRP_CUDA(launch_degrees(B->idx, B->nnz, pl->d.n_cols, pl->d_rank_b, pl->hot_R,
                                pl->d_items_b, pl->d_deg_b, pl->sm_count, s));
        pl->launches += 1;
    }
    return CRP_OK;
}

static void set_dense_args(crp_plan *pl, AccumulateArgs &a) {
    if (pl->hot_R) {
        a.hot_rank_a = pl->d_rank_a;
        a.hot_rank_b = pl->d_rank_b;
        a.hot_block = pl->d_hot;
        a.hot_R = pl->hot_R;
    }
    if (pl->warm_W) {
        a.warm_rank_a = pl->d_wrank_a;
        a.warm_rank_b = pl->d_wrank_b;
        a.warm_a = pl->d_warm_a;
        a.warm_b = pl->d_warm_b;
        a.warm_W = pl->warm_W;
        a.warm_in_hot = pl->warm_in_hot ? 1 : 0;
    }
}

static crp_status flush_dense(crp_plan *pl, const TableView &tv) {
    if (pl->hot_R) {
        CRP_CUDA(launch_hot_flush(pl->d_hot, pl->hot_R, pl->d_items_a, pl->d_items_b, pl->hp, tv,
                                  &pl->dc->flushed, pl->stream));
        pl->launches += 1;
    }
    if (pl->warm_W) {
        CRP_CUDA(launch_warm_flush(pl->d_warm_a, pl->warm_W, pl->d.n_cols, pl->d_witems_a, 1,
                                   pl->hp, tv, &pl->dc->flushed, pl->stream));
        CRP_CUDA(launch_warm_flush(pl->d_warm_b, pl->warm_W, pl->d.n_rows, pl->d_witems_b, 0,
                                   pl->hp, tv, &pl->dc->flushed, pl->stream));
        pl->launches += 2;
    }
    return CRP_OK;
}

extern "C" crp_status crp_outer_accumulate(crp_plan *pl, const crp_sparse *A, const crp_sparse *B) {
    if (!pl) return fail(CRP_EINVAL, "null plan");
    crp_status st = check_sparse(A, "A");
    if (st != CRP_OK) return st;
    st = check_sparse(B, "B");
    if (st != CRP_OK) return st;
    if (A->n_major != B->n_major)
        return fail(CRP_EINVAL, "A and B must hold the same number of outer products");
    if (A->n_minor != pl->d.n_rows || B->n_minor != pl->d.n_cols)
        return fail(CRP_EINVAL, "A->n_minor must equal n_rows and B->n_minor n_cols");
    if (pl->d.value_type == CRP_I32 && (A->val || B->val))
        return fail(CRP_EINVAL, "CRP_I32 counts {0,1} inputs: val must be NULL");
    if (A->n_major == 0) return CRP_OK;
    CRP_CUDA(cudaSetDevice(pl->device));
    if (pl->tune_first) {
        // P = 0: tune on this call's first outer products, then become that plan
        crp_plan_desc best;
        const int64_t sample = std::min<int64_t>(A->n_major, (int64_t)1 << 21);
        crp_status ts = crp_autotune(&pl->user_desc, A, B, sample, nullptr, &best, nullptr,
                                     (void *)pl->stream);
        if (ts != CRP_OK) return ts;
        crp_plan *fresh = nullptr;
        ts = crp_plan_create(&fresh, &best, (void *)pl->stream);
        if (ts != CRP_OK) return ts;
        std::swap(*pl, *fresh);
        crp_plan_destroy(fresh);   // the placeholder's buffers
    }
    if (pl->d.flags & CRP_PLAN_DEBUG_CHECKS) {
        unsigned int *bad = (unsigned int *)(pl->d_scratch64 + 2 * pl->d.P + 8);
        CRP_CUDA(cudaMemsetAsync(bad, 0, 4, pl->stream));
        CRP_CUDA(launch_validate_sparse(A->ptr, A->idx, A->n_major, A->nnz, A->n_minor, bad,
                                        pl->stream));
        CRP_CUDA(launch_validate_sparse(B->ptr, B->idx, B->n_major, B->nnz, B->n_minor, bad,
                                        pl->stream));
        unsigned int h_bad = 0;
        CRP_CUDA(cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, pl->stream));
        CRP_CUDA(cudaStreamSynchronize(pl->stream));
        if (h_bad) return fail(CRP_EINVAL, "input failed validation (ptr not monotone, "
                                           "ptr[K] != nnz, or an index out of range)");
    }
    const int32_t *b_idx = B->idx;
    const float *b_val = B->val;
    const uint32_t *b_hash = nullptr;
    if (pl->G > 1 && !(pl->d.flags & CRP_PLAN_ROUTED)) {
        st = ensure_sort_scratch(pl, B->nnz, B->n_major, B->val != nullptr);
        if (st != CRP_OK) return st;
        CRP_CUDA(launch_sort_by_hash(B->ptr, B->idx, B->val, B->n_major, pl->hp.hb, pl->s_idx,
                                     pl->s_val, pl->s_hash, pl->dc, pl->s_long, pl->sm_count,
                                     pl->stream));
        b_idx = pl->s_idx;
        b_val = B->val ? pl->s_val : nullptr;
        b_hash = pl->s_hash;
        pl->launches += 2;
    }
    if (!pl->tables_ready) {
        st = estimate_and_allocate(pl, A, B, b_idx, b_val);
        if (st != CRP_OK) return st;
    }
    if (pl->summary && !pl->locked) return summary_accumulate(pl, A, B);
    if (pl->d.flags & CRP_PLAN_ROUTED) return routed_accumulate(pl, A, B);
    AccumulateArgs a = make_args(pl, A, B, b_idx, b_val, pl->G);
    a.tv = table_view(pl, pl->slots, pl->d_off, pl->d_mask);
    if (pl->d.hot_items || pl->d.warm_items) {
        st = select_hot_items(pl, A, B);
        if (st == CRP_OK) st = count_degrees(pl, A, B);
        if (st != CRP_OK) return st;
        set_dense_args(pl, a);
    }
    CRP_CUDA(cudaMemsetAsync(&pl->dc->work_next, 0, sizeof(unsigned int), pl->stream));
    CRP_CUDA(cudaEventRecord(pl->ev0, pl->stream));
    CRP_CUDA(launch_accumulate(a, b_hash, pl->grid, pl->stream));
    st = flush_dense(pl, a.tv);
    if (st != CRP_OK) return st;
    CRP_CUDA(cudaEventRecord(pl->ev1, pl->stream));
    pl->timed = true;
    pl->timed_mid = false;
    pl->launches += 1;
    return CRP_OK;
}

// ---------------------------------------------------------------------------
// Sync, growth of full partitions
// ---------------------------------------------------------------------------

static crp_status grow_full_partitions(crp_plan *pl) {
    const uint32_t P = pl->d.P;
    for (int round = 0; round < 8; ++round) {
        std::vector<unsigned int> full(P);
        CRP_CUDA(cudaMemcpyAsync(full.data(), pl->d_full, P * 4, cudaMemcpyDeviceToHost,
                                 pl->stream));
        unsigned long long n_spill = 0;
        CRP_CUDA(cudaMemcpyAsync(&n_spill, &pl->dc->spill_n, 8, cudaMemcpyDeviceToHost,
                                 pl->stream));
        CRP_CUDA(cudaStreamSynchronize(pl->stream));
        if (n_spill > pl->spill_cap)
            return fail(CRP_ETABLE_FULL, "spill list overflowed; counts were lost (reset and "
                                         "create the plan with a larger table_capacity_hint)");
        bool any = false;
        for (auto f : full) any |= f != 0;
        if (!any && n_spill == 0) return CRP_OK;
        // new layout: full partitions x4
        std::vector<unsigned long long> noff(P), nmask(P);
        uint64_t total = 0;
        for (uint32_t p = 0; p < P; ++p) {
            uint64_t cap = pl->h_mask[p] + 1;
            if (full[p]) cap *= 4;
            noff[p] = total;
            nmask[p] = cap - 1;
            total += cap;
        }
        Slot *ns = nullptr;
        CRP_CUDA(cudaMalloc(&ns, total * sizeof(Slot)));
        CRP_CUDA(launch_fill_empty(ns, total, pl->stream));
        unsigned long long *d_noff = nullptr, *d_nmask = nullptr;
        CRP_CUDA(cudaMalloc(&d_noff, P * 8));
        CRP_CUDA(cudaMalloc(&d_nmask, P * 8));
        CRP_CUDA(cudaMemcpyAsync(d_noff, noff.data(), P * 8, cudaMemcpyHostToDevice, pl->stream));
        CRP_CUDA(cudaMemcpyAsync(d_nmask, nmask.data(), P * 8, cudaMemcpyHostToDevice, pl->stream));
        TableView tv = table_view(pl, ns, d_noff, d_nmask);
        for (uint32_t p = 0; p < P; ++p) {
            uint64_t cap = pl->h_mask[p] + 1;
            if (full[p])
                CRP_CUDA(launch_rehash_partition(pl->slots, pl->h_off[p], cap, tv, noff[p],
                                                 nmask[p], pl->stream));
            else
                CRP_CUDA(cudaMemcpyAsync(ns + noff[p], pl->slots + pl->h_off[p], cap * sizeof(Slot),
                                         cudaMemcpyDeviceToDevice, pl->stream));
        }
        // move the spill list aside and re-insert it into the grown tables
        SpillRec *old_spill = nullptr;
        if (n_spill) {
            CRP_CUDA(cudaMalloc(&old_spill, n_spill * sizeof(SpillRec)));
            CRP_CUDA(cudaMemcpyAsync(old_spill, pl->spill, n_spill * sizeof(SpillRec),
                                     cudaMemcpyDeviceToDevice, pl->stream));
        }
        CRP_CUDA(cudaMemsetAsync(&pl->dc->spill_n, 0, 8, pl->stream));
        CRP_CUDA(cudaMemsetAsync(pl->d_full, 0, P * 4, pl->stream));
        CRP_CUDA(cudaMemcpyAsync(pl->d_off, noff.data(), P * 8, cudaMemcpyHostToDevice, pl->stream));
        CRP_CUDA(cudaMemcpyAsync(pl->d_mask, nmask.data(), P * 8, cudaMemcpyHostToDevice,
                                 pl->stream));
        TableView tv2 = table_view(pl, ns, pl->d_off, pl->d_mask);
        if (n_spill) CRP_CUDA(launch_spill_reinsert(old_spill, n_spill, pl->hp, tv2, pl->stream));
        CRP_CUDA(cudaStreamSynchronize(pl->stream));
        cudaFree(old_spill);
        cudaFree(d_noff);
        cudaFree(d_nmask);
        cudaFree(pl->slots);
        pl->slots = ns;
        pl->n_slots = total;
        pl->h_off = noff;
        pl->h_mask = nmask;
    }
    return fail(CRP_ETABLE_FULL, "partitions still full after repeated growth");
}

extern "C" crp_status crp_sync(crp_plan *pl) {
    if (!pl) return fail(CRP_EINVAL, "null plan");
    crp_status ps = ensure_pinned(pl);
    if (ps != CRP_OK) return ps;
    // the status word comes back behind the stream's work: one round trip
    unsigned int *h_status = (unsigned int *)(pl->h_counts + 3);
    CRP_CUDA(cudaMemcpyAsync(h_status, &pl->dc->status, 4, cudaMemcpyDeviceToHost, pl->stream));
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    const unsigned int status = *h_status;
    if (status & kStatusBadIndex)
        return fail(CRP_EINVAL, "an input index was out of range (or a vector too long to sort)");
    if (status & kStatusNotOwned)
        return fail(CRP_ECUDA, "an update reached a partition outside the plan's interval");
    if (status & kStatusSmemProbe) return fail(CRP_ECUDA, "on-chip table probe bound exceeded");
    if (status & kStatusTimeout) return fail(CRP_ETIMEOUT, "a bounded device wait gave up");
    if (status & (kStatusTableFull | kStatusSpillFull)) {
        if (!pl->d.auto_grow || (status & kStatusSpillFull))
            return fail(CRP_ETABLE_FULL, (status & kStatusSpillFull)
                                             ? "spill list overflowed; counts were lost"
                                             : "a partition table is full (auto_grow is off)");
        crp_status st = grow_full_partitions(pl);
        if (st != CRP_OK) return st;
        unsigned int zero = 0;
        CRP_CUDA(cudaMemcpy(&pl->dc->status, &zero, 4, cudaMemcpyHostToDevice));
    }
    return CRP_OK;
}

// ---------------------------------------------------------------------------
// Top-k, export, stats
// ---------------------------------------------------------------------------

static bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// The k heaviest of n_c candidates (an MSD radix select first when more than
// one CTA can sort), sorted and written out; *n_out = entries written and
// *kth_w (nullable) = the weight of the last one.  cand stays the caller's.
// Grow a plan-owned scratch buffer (kept across calls: an allocation and a
// free per top-k call would each synchronise the device).
template <typename T>
static crp_status plan_scratch(T *&buf, uint64_t &cap, uint64_t need) {
    if (need <= cap) return CRP_OK;
    cudaFree(buf);
    buf = nullptr;
    cap = 0;
    CRP_CUDA(cudaMalloc(&buf, need * sizeof(T)));
    cap = need;
    return CRP_OK;
}

static crp_status topk_from_candidates(crp_plan *pl, const TopkCand *cand, uint64_t n_c, int32_t k,
                                       int32_t *i_out, int32_t *j_out, double *w_out,
                                       double *w_lower, int32_t *n_out, double *kth_w) {
    cudaStream_t s = pl->stream;
    unsigned int *cnt = pl->d_topk_hist + kTopkBuckets;  // 3 counters + 256-bin hist after
    unsigned int *dhist = cnt + 4;
    crp_status st = CRP_OK;
    auto cuda_ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == CRP_OK)
            st = fail(CRP_ECUDA, std::string("topk: ") + cudaGetErrorString(e));
        return st == CRP_OK;
    };
    const TopkCand *final_c = cand;
    unsigned int final_sort = (unsigned int)n_c;  // candidates to sort
    unsigned int final_n = (unsigned int)std::min<uint64_t>(n_c, (uint64_t)k);
    if (n_c > (uint64_t)kTopkSortMax) {
        st = plan_scratch(pl->d_cand_keep, pl->cand_keep_cap, n_c);
        if (st == CRP_OK) st = plan_scratch(pl->d_cand_sel, pl->cand_sel_cap, (uint64_t)kTopkSortMax);
        if (st != CRP_OK) return st;
        TopkCand *sel = pl->d_cand_sel, *keep = pl->d_cand_keep;
        // first cut: the candidates at or above the log-linear bucket that
        // holds the k-th largest weight (usually a few more than k)
        std::vector<unsigned int> hist(kTopkBuckets);
        cuda_ok(launch_cand_hist(cand, (unsigned int)n_c, pl->d_topk_hist, s));
        cuda_ok(cudaMemcpyAsync(hist.data(), pl->d_topk_hist, kTopkBuckets * 4,
                                cudaMemcpyDeviceToHost, s));
        cuda_ok(cudaStreamSynchronize(s));
        if (st != CRP_OK) return st;
        uint64_t cum = 0;
        int b = kTopkBuckets - 1;
        for (; b > 0; --b) {
            cum += hist[b];
            if (cum >= (uint64_t)k) break;
        }
        cuda_ok(launch_cand_collect(cand, (unsigned int)n_c, (unsigned int)b, keep, cnt + 2, s));
        pl->launches += 2;
        unsigned int n1 = 0;
        cuda_ok(cudaMemcpyAsync(&n1, cnt + 2, 4, cudaMemcpyDeviceToHost, s));
        cuda_ok(cudaStreamSynchronize(s));
        if (st != CRP_OK) return st;
        final_c = keep;
        final_sort = n1;
        final_n = std::min<unsigned int>(n1, (unsigned int)k);
        if (n1 > (unsigned int)kTopkSortMax) {
            // MSD radix select on the remaining candidates down to exactly k
            // (the collected ones move between keep and cand_tmp)
            st = plan_scratch(pl->d_cand_tmp, pl->cand_tmp_cap, (uint64_t)n1);
            if (st != CRP_OK) return st;
            TopkCand *und = keep, *nxt = pl->d_cand_tmp;
            unsigned int n_und = n1, n_sel = 0, need = (unsigned int)k;
            cuda_ok(cudaMemsetAsync(cnt + 1, 0, 4, s));  // sel count
            for (int d = 0; d < 16 && st == CRP_OK && need > 0; ++d) {
                unsigned int h[256];
                cuda_ok(launch_topk_digit_hist(und, n_und, d, dhist, s));
                cuda_ok(cudaMemcpyAsync(h, dhist, sizeof h, cudaMemcpyDeviceToHost, s));
                cuda_ok(cudaStreamSynchronize(s));
                if (st != CRP_OK) break;
                unsigned int above = 0;
                int pivot = 255;
                for (; pivot >= 0; --pivot) {
                    if (above + h[pivot] >= need) break;
                    above += h[pivot];
                }
                if (above == 0 && h[pivot] == n_und) continue;   // one digit value: next digit
                cuda_ok(launch_topk_digit_split(und, n_und, d, (unsigned)pivot, sel, cnt + 1, nxt,
                                                cnt + 2, s));
                pl->launches += 2;
                unsigned int kn = 0;
                cuda_ok(cudaMemcpyAsync(&kn, cnt + 2, 4, cudaMemcpyDeviceToHost, s));
                cuda_ok(cudaStreamSynchronize(s));
                n_sel += above;
                need -= above;
                std::swap(und, nxt);
                n_und = kn;
                if (n_und == need) {  // everything left at this prefix is in
                    cuda_ok(cudaMemcpyAsync(sel + n_sel, und, (size_t)n_und * sizeof(TopkCand),
                                            cudaMemcpyDeviceToDevice, s));
                    n_sel += n_und;
                    need = 0;
                }
            }
            final_c = sel;
            final_n = n_sel;
            final_sort = n_sel;
        }
    }
    // write out (through a device staging buffer when the outputs are host memory)
    const bool dev_out = is_device_ptr(i_out);
    int32_t *di = i_out, *dj = j_out;
    double *dw = w_out, *dwl = w_lower;
    if (st == CRP_OK && !dev_out) {
        st = plan_scratch(pl->d_topk_stage, pl->topk_stage_cap,
                          (uint64_t)kTopkSortMax * (4 + 4 + 8 + 8));
        if (st != CRP_OK) return st;
        di = (int32_t *)pl->d_topk_stage;
        dj = di + k;
        dw = (double *)(dj + k);
        dwl = w_lower ? dw + k : nullptr;
    }
    if (st == CRP_OK)
        cuda_ok(launch_topk_sort_write(final_c, final_sort, final_n, di, dj, dw, dwl, s));
    pl->launches += 1;
    if (st == CRP_OK && !dev_out) {
        cuda_ok(cudaMemcpyAsync(i_out, di, final_n * 4, cudaMemcpyDeviceToHost, s));
        cuda_ok(cudaMemcpyAsync(j_out, dj, final_n * 4, cudaMemcpyDeviceToHost, s));
        cuda_ok(cudaMemcpyAsync(w_out, dw, final_n * 8, cudaMemcpyDeviceToHost, s));
        if (w_lower) cuda_ok(cudaMemcpyAsync(w_lower, dwl, final_n * 8, cudaMemcpyDeviceToHost, s));
    }
    if (st == CRP_OK && kth_w && final_n)
        cuda_ok(cudaMemcpyAsync(kth_w, dw + (final_n - 1), 8, cudaMemcpyDeviceToHost, s));
    cuda_ok(cudaStreamSynchronize(s));
    if (st == CRP_OK) *n_out = (int32_t)final_n;
    return st;
}


// Top k certified from the hot block ({0,1} inputs, exact tables, a hot set):
// the hot pairs present in the tables are the candidates, and their top k is
// the answer when its k-th weight is above every degree outside the hot set
// (each entry is at most the smaller degree of its row and column, so no
// entry outside the hot block can reach it).  *done = false when the bound
// does not hold or there are fewer than k candidates: the caller then scans
// the tables.
static crp_status topk_certified(crp_plan *pl, int32_t k, int upper, int32_t *i_out,
                                 int32_t *j_out, double *w_out, double *w_lower, int32_t *n_out,
                                 bool *done) {
    *done = false;
    const uint32_t R = pl->hot_R;
    cudaStream_t s = pl->stream;
    if (!pl->d_hot_cand)
        CRP_CUDA(cudaMalloc(&pl->d_hot_cand, (size_t)R * R * sizeof(TopkCand)));
    unsigned int *count = pl->d_topk_hist + kTopkBuckets + 3;
    unsigned long long *bound = pl->d_scratch64 + 2 * (size_t)pl->d.P + 10;
    CRP_CUDA(cudaMemsetAsync(bound, 0, 8, s));
    CRP_CUDA(launch_topk_hot_candidates(pl->slots, pl->d_off, pl->d_mask, pl->hp, pl->d_items_a,
                                        pl->d_items_b, R, upper, pl->d_hot_cand, count, s));
    CRP_CUDA(launch_max_outside(pl->d_deg_a, pl->d.n_rows, pl->d_rank_a, R, bound, s));
    CRP_CUDA(launch_max_outside(pl->deg_b_mirrors_a ? pl->d_deg_a : pl->d_deg_b, pl->d.n_cols,
                                pl->d_rank_b, R, bound, s));
    pl->launches += 3;
    unsigned int n_c = 0;
    unsigned long long S = 0;
    CRP_CUDA(cudaMemcpyAsync(&n_c, count, 4, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaMemcpyAsync(&S, bound, 8, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaStreamSynchronize(s));
    if (n_c < (unsigned int)k) return CRP_OK;
    double kth = 0.0;
    int32_t n = 0;
    crp_status st = topk_from_candidates(pl, pl->d_hot_cand, n_c, k, i_out, j_out, w_out, w_lower,
                                         &n, &kth);
    if (st != CRP_OK) return st;
    if (n == k && kth > (double)S) {
        *n_out = n;
        *done = true;
        pl->topk_certified += 1;
    }
    return CRP_OK;
}

extern "C" crp_status crp_topk(crp_plan *pl, int32_t k, uint32_t flags, int32_t *i_out,
                               int32_t *j_out, double *w_out, double *w_lower, int32_t *n_out) {
    if (!pl || !i_out || !j_out || !w_out || !n_out) return fail(CRP_EINVAL, "null argument");
    if (k < 1 || k > kTopkSortMax) return fail(CRP_EINVAL, "k must be in [1, 8192]");
    *n_out = 0;
    if (!pl->tables_ready) return CRP_OK;
    const int upper = (flags & CRP_TOPK_UPPER) ? 1 : 0;
    if (!pl->summary && pl->d.value_type == CRP_I32 && pl->hot_R && pl->d_deg_a) {
        bool done = false;
        crp_status cs = topk_certified(pl, k, upper, i_out, j_out, w_out, w_lower, n_out, &done);
        if (cs != CRP_OK || done) return cs;
    }
    cudaStream_t s = pl->stream;
    const int vt = pl->summary ? kVTSummary : pl->d.value_type;
    unsigned int *cnt = pl->d_topk_hist + kTopkBuckets;  // collected-candidate counter
    // candidates: the slots at or above a histogram bucket.  A large table is
    // first tried with a 1/32 sample histogram and a bucket expected to hold
    // about 2k + 256 slots; k or more collected slots at or above a bucket
    // contain the top k, otherwise the exact histogram decides.
    const int shift = pl->n_slots >= (1ull << 26) ? 5 : 0;
    TopkCand *cand = nullptr;
    uint64_t n_c = 0;
    std::vector<unsigned int> hist(kTopkBuckets);
    for (int sh : {shift, 0}) {
        CRP_CUDA(launch_topk_hist(pl->slots, pl->n_slots, vt, upper, sh, pl->d_topk_hist, s));
        pl->launches += 1;
        CRP_CUDA(cudaMemcpyAsync(hist.data(), pl->d_topk_hist, kTopkBuckets * 4,
                                 cudaMemcpyDeviceToHost, s));
        CRP_CUDA(cudaStreamSynchronize(s));
        const uint64_t want = sh ? (((uint64_t)2 * k + 256) >> sh) + 1 : (uint64_t)k;
        uint64_t cum = 0;
        int b = kTopkBuckets - 1;
        for (; b >= 0; --b) {
            cum += hist[b];
            if (cum >= want) break;
        }
        if (b < 0) {
            if (sh) continue;   // the sample holds too few slots: take the exact histogram
            b = 0;
        }
        if (cum == 0) break;
        // capacity: the exact count, or twice the sampled estimate plus slack
        const uint64_t cap = sh ? (cum << sh) * 2 + 4 * (uint64_t)k + 1024 : cum;
        cudaFree(cand);
        if (cap > 0xffffffffull) return fail(CRP_EUNSUPPORTED, "too many top-k candidates");
        cand = nullptr;
        CRP_CUDA(cudaMalloc(&cand, cap * sizeof(TopkCand)));
        CRP_CUDA(launch_topk_collect(pl->slots, pl->n_slots, vt, upper, (unsigned)b, cand, cnt,
                                     (unsigned)cap, s));
        pl->launches += 1;
        if (sh == 0) {   // the exact histogram already counted the candidates
            n_c = cum;
            break;
        }
        unsigned int got = 0;
        CRP_CUDA(cudaMemcpyAsync(&got, cnt, 4, cudaMemcpyDeviceToHost, s));
        CRP_CUDA(cudaStreamSynchronize(s));
        n_c = got;
        if (got >= (unsigned)k && got <= cap) break;
        n_c = 0;
    }
    if (n_c == 0) {
        cudaFree(cand);
        return CRP_OK;
    }
    crp_status fs = topk_from_candidates(pl, cand, n_c, k, i_out, j_out, w_out, w_lower, n_out,
                                         nullptr);
    cudaFree(cand);
    return fs;
}

extern "C" uint64_t crp_topk_certified_calls(const crp_plan *pl) {
    return pl ? pl->topk_certified : 0;
}

extern "C" crp_status crp_export_partitions(crp_plan *pl, uint32_t p0, uint32_t p1, int32_t *i_out,
                                            int32_t *j_out, double *w_out, double *w_lower,
                                            int64_t capacity, int64_t *n_out) {
    if (!pl || !n_out) return fail(CRP_EINVAL, "null argument");
    if (p0 > p1 || p1 > pl->d.P) return fail(CRP_EINVAL, "bad partition range");
    *n_out = 0;
    if (!pl->tables_ready || p0 == p1) return CRP_OK;
    const uint32_t P = pl->d.P;
    cudaStream_t s = pl->stream;
    unsigned long long *d_terms = pl->d_scratch64, *d_live = pl->d_scratch64 + P;
    CRP_CUDA(launch_partition_sums(pl->slots, pl->d_off, pl->d_mask, P, pl->d.value_type, d_terms,
                                   d_live, s));
    std::vector<unsigned long long> live(P);
    CRP_CUDA(cudaMemcpyAsync(live.data(), d_live, P * 8, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaStreamSynchronize(s));
    std::vector<unsigned long long> base(p1 - p0);
    unsigned long long tot = 0;
    for (uint32_t p = p0; p < p1; ++p) {
        base[p - p0] = tot;
        tot += live[p];
    }
    *n_out = (int64_t)tot;
    if ((int64_t)tot > capacity) return fail(CRP_EINVAL, "export capacity too small");
    if (tot == 0) return CRP_OK;
    if (!i_out || !j_out || !w_out) return fail(CRP_EINVAL, "null output");
    const bool dev_out = is_device_ptr(i_out);
    unsigned long long *d_base = nullptr;
    CRP_CUDA(cudaMalloc(&d_base, base.size() * 8));
    CRP_CUDA(cudaMemcpyAsync(d_base, base.data(), base.size() * 8, cudaMemcpyHostToDevice, s));
    int32_t *di = i_out, *dj = j_out;
    double *dw = w_out, *dwl = w_lower;
    void *stage = nullptr;
    if (!dev_out) {
        CRP_CUDA(cudaMalloc(&stage, tot * (4 + 4 + 8 + 8)));
        di = (int32_t *)stage;
        dj = di + tot;
        dw = (double *)(dj + tot);
        dwl = w_lower ? dw + tot : nullptr;
    }
    CRP_CUDA(launch_export_range(pl->slots, pl->d_off, pl->d_mask, p0, p1, d_base,
                                 pl->summary ? kVTSummary : pl->d.value_type, di, dj, dw, dwl, s));
    if (!dev_out) {
        CRP_CUDA(cudaMemcpyAsync(i_out, di, tot * 4, cudaMemcpyDeviceToHost, s));
        CRP_CUDA(cudaMemcpyAsync(j_out, dj, tot * 4, cudaMemcpyDeviceToHost, s));
        CRP_CUDA(cudaMemcpyAsync(w_out, dw, tot * 8, cudaMemcpyDeviceToHost, s));
        if (w_lower) CRP_CUDA(cudaMemcpyAsync(w_lower, dwl, tot * 8, cudaMemcpyDeviceToHost, s));
    }
    CRP_CUDA(cudaStreamSynchronize(s));
    cudaFree(stage);
    cudaFree(d_base);
    return CRP_OK;
}

extern "C" crp_status crp_stats(crp_plan *pl, crp_stats_t *out, uint64_t *terms_out) {
    if (!pl || !out) return fail(CRP_EINVAL, "null argument");
    memset(out, 0, sizeof *out);
    const uint32_t P = pl->d.P;
    out->P = P;
    cudaStream_t s = pl->stream;
    DevCounters dc;
    CRP_CUDA(cudaMemcpyAsync(&dc, pl->dc, sizeof dc, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaStreamSynchronize(s));
    out->terms = dc.terms;
    out->flushed_updates = dc.flushed;
    out->spilled = dc.spill_n;
    out->table_slots = pl->n_slots;
    out->launches = pl->launches;
    out->estimated_entries = pl->est_entries;
    if (pl->timed) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pl->ev0, pl->ev1) == cudaSuccess) out->last_accumulate_ms = ms;
        else cudaGetLastError();
        if (pl->timed_mid && cudaEventElapsedTime(&ms, pl->ev0, pl->evm) == cudaSuccess)
            out->last_route_ms = ms;
        else cudaGetLastError();
    }
    if (!pl->tables_ready) return CRP_OK;
    unsigned long long *d_terms = pl->d_scratch64, *d_live = pl->d_scratch64 + P;
    CRP_CUDA(launch_partition_sums(pl->slots, pl->d_off, pl->d_mask, P, pl->d.value_type, d_terms,
                                   d_live, s));
    std::vector<unsigned long long> terms(P), live(P);
    std::vector<unsigned int> full(P);
    CRP_CUDA(cudaMemcpyAsync(terms.data(), d_terms, P * 8, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaMemcpyAsync(live.data(), d_live, P * 8, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaMemcpyAsync(full.data(), pl->d_full, P * 4, cudaMemcpyDeviceToHost, s));
    CRP_CUDA(cudaStreamSynchronize(s));
    unsigned long long mx = 0, sum = 0;
    for (uint32_t p = 0; p < P; ++p) {
        out->entries += live[p];
        out->full_partitions += full[p] ? 1 : 0;
        mx = std::max(mx, terms[p]);
        sum += terms[p];
        if (terms_out) terms_out[p] = terms[p];
    }
    out->max_over_mean_terms = sum ? (double)mx / ((double)sum / P) : 0.0;
    return CRP_OK;
}

extern "C" crp_status crp_timing(crp_plan *pl, double *accumulate_ms, uint64_t *launches) {
    if (!pl) return fail(CRP_EINVAL, "null plan");
    if (launches) *launches = pl->launches;
    if (accumulate_ms) {
        *accumulate_ms = pl->summary ? pl->summary_ms : 0.0;
        if (pl->timed) {
            CRP_CUDA(cudaEventSynchronize(pl->ev1));
            float ms = 0.f;
            CRP_CUDA(cudaEventElapsedTime(&ms, pl->ev0, pl->ev1));
            *accumulate_ms = ms;
        }
    }
    return CRP_OK;
}

// A ragged block over the reserved pairs: rows are the items i of reserved
// keys and columns the items j, each side ranked by how many reserved keys
// hold it; row r spans the columns up to its last reserved one, so a pair
// of a reserved row lies in the block when its column's rank is below the
// row's length (one comparison per term).  Cells of reserved pairs count
// them during accumulation; the other cells are off, and their pairs take
// the summary path as before.  The block is added into the reserved counters
// at the end of each call.  A reserved pair then costs a dense atomic instead
// of a hash probe, and the rest of the stream skips the reserved-key test.
static crp_status reserve_dense_block(crp_plan *pl) {
    std::vector<unsigned long long> keys(pl->n_res);
    CRP_CUDA(cudaMemcpyAsync(keys.data(), pl->d_res_keys, pl->n_res * 8, cudaMemcpyDeviceToHost,
                             pl->stream));
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    pl->resv_rows = 0;
    pl->resv_cells = 0;
    std::unordered_map<uint32_t, uint32_t> deg_a, deg_b;
    for (auto k : keys) {
        ++deg_a[(uint32_t)(k >> 32)];
        ++deg_b[(uint32_t)k];
    }
    if (deg_a.empty() || deg_a.size() >= 0xFFFF || deg_b.size() >= 0xFFFF) return CRP_OK;
    auto ranked = [](const std::unordered_map<uint32_t, uint32_t> &deg) {
        std::vector<std::pair<uint32_t, uint32_t>> v(deg.begin(), deg.end());
        std::sort(v.begin(), v.end(), [](const auto &x, const auto &y) {
            return x.second != y.second ? x.second > y.second : x.first < y.first;
        });
        return v;
    };
    const auto rows = ranked(deg_a), cols = ranked(deg_b);
    std::unordered_map<uint32_t, uint32_t> ra, rb;
    for (uint32_t r = 0; r < rows.size(); ++r) ra[rows[r].first] = r;
    for (uint32_t c = 0; c < cols.size(); ++c) rb[cols[c].first] = c;
    std::vector<unsigned int> len(rows.size(), 0), off(rows.size(), 0), idx(keys.size());
    for (auto k : keys) {
        unsigned int &l = len[ra[(uint32_t)(k >> 32)]];
        l = std::max<unsigned int>(l, rb[(uint32_t)k] + 1);
    }
    uint64_t total = 0;
    for (size_t r = 0; r < rows.size(); ++r) {
        off[r] = (unsigned int)total;
        total += len[r];
    }
    if (total > (64ull << 20)) return CRP_OK;   // too sparse a block: keep the hash probe
    for (size_t x = 0; x < keys.size(); ++x)
        idx[x] = off[ra[(uint32_t)(keys[x] >> 32)]] + rb[(uint32_t)keys[x]];
    std::vector<int64_t> ia(rows.size()), ib(cols.size());
    for (size_t r = 0; r < rows.size(); ++r) ia[r] = rows[r].first;
    for (size_t c = 0; c < cols.size(); ++c) ib[c] = cols[c].first;
    cudaFree(pl->d_hot);
    cudaFree(pl->d_items_a);
    cudaFree(pl->d_items_b);
    cudaFree(pl->d_resv_len);
    cudaFree(pl->d_resv_off);
    cudaFree(pl->d_resv_idx);
    pl->d_hot = nullptr;
    pl->d_items_a = pl->d_items_b = nullptr;
    pl->d_resv_len = pl->d_resv_off = pl->d_resv_idx = nullptr;
    CRP_CUDA(cudaMalloc(&pl->d_hot, std::max<uint64_t>(total, 1) * 4));
    CRP_CUDA(cudaMalloc(&pl->d_items_a, ia.size() * 8));
    CRP_CUDA(cudaMalloc(&pl->d_items_b, ib.size() * 8));
    CRP_CUDA(cudaMalloc(&pl->d_resv_len, len.size() * 4));
    CRP_CUDA(cudaMalloc(&pl->d_resv_off, off.size() * 4));
    CRP_CUDA(cudaMalloc(&pl->d_resv_idx, idx.size() * 4));
    CRP_CUDA(cudaMemcpyAsync(pl->d_items_a, ia.data(), ia.size() * 8, cudaMemcpyHostToDevice,
                             pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_items_b, ib.data(), ib.size() * 8, cudaMemcpyHostToDevice,
                             pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_resv_len, len.data(), len.size() * 4, cudaMemcpyHostToDevice,
                             pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_resv_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice,
                             pl->stream));
    CRP_CUDA(cudaMemcpyAsync(pl->d_resv_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice,
                             pl->stream));
    if (!pl->d_rank_a) {
        CRP_CUDA(cudaMalloc(&pl->d_rank_a, (size_t)pl->d.n_rows * 2));
        CRP_CUDA(cudaMalloc(&pl->d_rank_b, (size_t)pl->d.n_cols * 2));
    }
    CRP_CUDA(launch_hot_ranks(pl->d_rank_a, pl->d.n_rows, pl->d_items_a, (uint32_t)ia.size(),
                              pl->stream));
    CRP_CUDA(launch_hot_ranks(pl->d_rank_b, pl->d.n_cols, pl->d_items_b, (uint32_t)ib.size(),
                              pl->stream));
    CRP_CUDA(launch_reserve_cells(pl->d_resv_idx, (int32_t)idx.size(), pl->d_hot, total,
                                  pl->stream));
    pl->launches += 5;
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    pl->resv_rows = (uint32_t)rows.size();
    pl->resv_cells = total;
    return CRP_OK;
}

extern "C" crp_status crp_reserve(crp_plan *pl, const uint64_t *keys, int32_t n) {
    if (!pl || (n > 0 && !keys) || n < 0) return fail(CRP_EINVAL, "bad argument");
    if (!pl->summary || !pl->d.reserved_counters)
        return fail(CRP_EINVAL, "the plan has no reserved counters (summary mode only)");
    if ((int64_t)pl->n_res + n > (int64_t)pl->d.reserved_counters)
        return fail(CRP_EINVAL, "more keys than reserved_counters");
    if (n == 0) return CRP_OK;
    const bool dev = is_device_ptr(keys);
    CRP_CUDA(cudaMemcpyAsync(pl->d_res_keys + pl->n_res, keys, (size_t)n * 8,
                             dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, pl->stream));
    CRP_CUDA(launch_reserve_insert(pl->slots, pl->res_off, pl->res_mask, pl->d_res_keys + pl->n_res,
                                   n, pl->stream));
    CRP_CUDA(launch_reserve_bits(pl->d_res_keys + pl->n_res, n, pl->d_res_bits,
                                 pl->d_res_bits + (pl->d.n_rows + 31) / 32, pl->stream));
    pl->launches += 2;
    pl->n_res += n;
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    return reserve_dense_block(pl);
}

// ---------------------------------------------------------------------------
// Count-Sketch (Preliminaries; Figure 1)
// ---------------------------------------------------------------------------

extern "C" crp_status crp_sketch_read(crp_plan *pl, void *out) {
    if (!pl || !out) return fail(CRP_EINVAL, "null argument");
    if (!pl->d_sketch) return fail(CRP_EINVAL, "the plan keeps no sketch (CRP_PLAN_SKETCH)");
    CRP_CUDA(cudaSetDevice(pl->device));
    CRP_CUDA(cudaMemcpyAsync(out, pl->d_sketch, (size_t)pl->d.P * 8, cudaMemcpyDefault,
                             pl->stream));
    CRP_CUDA(cudaStreamSynchronize(pl->stream));
    return CRP_OK;
}

extern "C" crp_status crp_sketch_estimate(crp_plan *const *plans, int32_t t, const int32_t *i,
                                          const int32_t *j, int64_t n, double *out) {
    if (!plans || t < 1 || t > kSketchMaxT || n < 0 || (n > 0 && (!i || !j || !out)))
        return fail(CRP_EINVAL, "bad argument (1 <= t <= 32, n >= 0, device arrays)");
    SketchSet S;
    memset(&S, 0, sizeof(S));
    S.t = t;
    const crp_plan *p0 = plans[0];
    if (!p0) return fail(CRP_EINVAL, "null plan");
    S.value_type = p0->d.value_type;
    for (int32_t r = 0; r < t; ++r) {
        const crp_plan *pl = plans[r];
        if (!pl || !pl->d_sketch)
            return fail(CRP_EINVAL, "every plan must keep a sketch (CRP_PLAN_SKETCH)");
        if (pl->d.P != p0->d.P || pl->d.n_rows != p0->d.n_rows || pl->d.n_cols != p0->d.n_cols ||
            pl->d.value_type != p0->d.value_type || pl->device != p0->device)
            return fail(CRP_EINVAL, "the plans differ in P, shape, value type or device");
        S.hp[r] = pl->hp;
        S.sg[r] = pl->sg;
        S.cs[r] = pl->d_sketch;
    }
    if (n == 0) return CRP_OK;
    CRP_CUDA(cudaSetDevice(p0->device));
    for (int32_t r = 1; r < t; ++r)
        if (plans[r]->stream != p0->stream) CRP_CUDA(cudaStreamSynchronize(plans[r]->stream));
    unsigned int *bad = (unsigned int *)(p0->d_scratch64 + 2 * p0->d.P + 8);
    CRP_CUDA(cudaMemsetAsync(bad, 0, 4, p0->stream));
    CRP_CUDA(launch_sketch_estimate(S, i, j, n, p0->d.n_rows, p0->d.n_cols, out, bad,
                                    p0->stream));
    plans[0]->launches += 1;
    unsigned int h_bad = 0;
    CRP_CUDA(cudaMemcpyAsync(&h_bad, bad, 4, cudaMemcpyDeviceToHost, p0->stream));
    CRP_CUDA(cudaStreamSynchronize(p0->stream));
    if (h_bad) return fail(CRP_EINVAL, "an index lies outside [0, n_rows) x [0, n_cols)");
    return CRP_OK;
}
