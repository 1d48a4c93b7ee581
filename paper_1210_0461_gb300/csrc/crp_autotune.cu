// Launch-configuration autotuner.  It times candidate configurations of the
// exact product (partition count P, variant: on-chip combining table / direct
// HBM updates / routed two-phase with bins derived from the table size, dense
// tiers: hot blocks of 1024 or 4096 items, or 2048 items plus warm stripes of
// 32 or 64 items, tile of outer products per work item) on a prefix of the caller's
// outer products, and keeps the fastest.  Results are cached in a text file
// keyed by device name and a shape class of the input (log2 buckets of K,
// n_rows, n_cols and of the mean terms per outer product, plus value type and
// mode), one "key value..." line per entry.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <cmath>
#include <string>
#include <vector>

#include "crp_internal.cuh"

using namespace crp;

static int ilog2u(uint64_t x) {
    int l = 0;
    while (x > 1) { x >>= 1; ++l; }
    return l;
}

static std::string shape_key(const crp_plan_desc &d, int64_t K, double mean_terms) {
    cudaDeviceProp prop;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaGetDeviceProperties(&prop, dev);
    std::string name = prop.name;
    for (auto &c : name) if (c == ' ') c = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "%s:K%d:R%d:C%d:T%d:v%d:m%d", name.c_str(), ilog2u((uint64_t)K),
             ilog2u((uint64_t)d.n_rows), ilog2u((uint64_t)d.n_cols),
             ilog2u((uint64_t)(mean_terms + 1)), d.value_type, d.mode);
    return buf;
}

static bool cache_lookup(const char *path, const std::string &key, crp_plan_desc *out,
                         double *tps) {
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        char k[256];
        unsigned P, groups, tile, slots, flags, hot, warm;
        double v;
        if (sscanf(line, "%255s %u %u %u %u %u %u %u %lf", k, &P, &groups, &tile, &slots, &flags,
                   &hot, &warm, &v) == 9 && key == k) {
            out->P = P;
            out->hot_items = hot;
            out->warm_items = warm;
            out->groups = groups;
            out->tile_vectors = tile;
            out->smem_slots = slots;
            out->flags = flags;
            if (tps) *tps = v;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void cache_store(const char *path, const std::string &key, const crp_plan_desc &d,
                        double tps) {
    if (!path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %u %u %u %u %u %u %u %.17g\n", key.c_str(), d.P, d.groups, d.tile_vectors,
            d.smem_slots, d.flags, d.hot_items, d.warm_items, tps);
    fclose(f);
}

extern "C" crp_status crp_autotune(const crp_plan_desc *base, const crp_sparse *A,
                                   const crp_sparse *B, int64_t sample_vectors,
                                   const char *cache_path, crp_plan_desc *best,
                                   double *best_terms_per_s, void *stream) {
    if (!base || !A || !B || !best || A->n_major != B->n_major) {
        set_last_error("crp_autotune: bad argument");
        return CRP_EINVAL;
    }
    *best = *base;
    const int64_t K = A->n_major;
    const int64_t Ks = sample_vectors > 0 && sample_vectors < K ? sample_vectors : K;
    crp_sparse As = *A, Bs = *B;
    As.n_major = Bs.n_major = Ks;
    // terms of the sample (for the shape class and the rate)
    int64_t ptr_a[2], ptr_b[2];
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d_terms = nullptr;
    if (cudaMalloc(&d_terms, 8) != cudaSuccess) return CRP_ENOMEM;
    launch_count_terms(A->ptr, B->ptr, Ks, d_terms, s);
    unsigned long long terms = 0;
    cudaMemcpyAsync(&terms, d_terms, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(ptr_a, A->ptr + Ks, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(ptr_b, B->ptr + Ks, 8, cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    cudaFree(d_terms);
    if (e != cudaSuccess) {
        set_last_error(std::string("crp_autotune: ") + cudaGetErrorString(e));
        return CRP_ECUDA;
    }
    As.nnz = ptr_a[0];
    Bs.nnz = ptr_b[0];
    const std::string key = shape_key(*base, K, Ks ? (double)terms / (double)Ks : 0.0);
    if (cache_lookup(cache_path, key, best, best_terms_per_s)) return CRP_OK;

    struct Cand { uint32_t P, groups, tile, slots, flags, hot, warm; };
    std::vector<Cand> cands;
    const uint32_t Ps[] = {256, 1024, 4096};
    const uint32_t tiles[] = {32, 64, 256};
    const bool ints = base->value_type == CRP_I32;
    for (uint32_t P : Ps) {
        for (uint32_t t : tiles) cands.push_back({P, 1, t, 8192, CRP_PLAN_DIRECT, 0, 0});
        cands.push_back({P, 1, 64, 8192, 0u, 0, 0});
        cands.push_back({P, 1, 64, 16384, 0u, 0, 0});
        cands.push_back({P, 0, 64, 8192, CRP_PLAN_ROUTED, 0, 0});
        if (ints) {
            // hot block alone, and a smaller hot block with warm stripes
            const uint32_t tiers[4][2] = {{1024u, 0u}, {4096u, 0u}, {2048u, 32u}, {2048u, 64u}};
            // routed bins are left to the plan (groups = 0): it sizes them by
            // the table, which grows with the input, so a choice made on a
            // prefix carries over to the whole input
            for (const auto &hw : tiers) {
                cands.push_back({P, 1, 64, 8192, CRP_PLAN_DIRECT, hw[0], hw[1]});
                cands.push_back({P, 0, 64, 8192, CRP_PLAN_ROUTED, hw[0], hw[1]});
            }
        }
    }
    double best_tps = -1.0;
    for (const Cand &c : cands) {
        if (c.P > (uint32_t)std::max(base->n_rows, 1) * 64u && c.P > 256) continue;
        crp_plan_desc d = *base;
        d.P = c.P;
        d.groups = c.groups;
        d.tile_vectors = c.tile;
        d.smem_slots = c.slots;
        d.flags = (base->flags & ~(CRP_PLAN_DIRECT | CRP_PLAN_ROUTED)) | c.flags;
        d.hot_items = c.hot;
        d.warm_items = c.warm;
        d.table_capacity_hint = 0;
        d.auto_grow = 1;
        crp_plan *pl = nullptr;
        if (crp_plan_create(&pl, &d, stream) != CRP_OK) continue;
        double ms_best = 1e30;
        bool ok = true;
        for (int rep = 0; rep < 3 && ok; ++rep) {
            ok = crp_reset(pl) == CRP_OK && crp_outer_accumulate(pl, &As, &Bs) == CRP_OK &&
                 crp_sync(pl) == CRP_OK;
            double ms = 0;
            if (ok && rep > 0 && crp_timing(pl, &ms, nullptr) == CRP_OK && ms > 0)
                ms_best = std::min(ms_best, ms);
        }
        crp_plan_destroy(pl);
        if (!ok || ms_best >= 1e29) continue;
        const double tps = (double)terms / (ms_best * 1e-3);
        if (tps > best_tps) {
            best_tps = tps;
            *best = d;
            best->table_capacity_hint = base->table_capacity_hint;
            best->auto_grow = base->auto_grow;
        }
    }
    if (best_tps < 0) {
        set_last_error("crp_autotune: no candidate configuration ran");
        return CRP_ECUDA;
    }
    if (best_terms_per_s) *best_terms_per_s = best_tps;
    cache_store(cache_path, key, *best, best_tps);
    return CRP_OK;
}

// Batched products: the partition count and the outer products per work item
// of the one persistent launch, timed on a sample of the problems (every
// stride-th problem, so the sample spans the batch's sizes).  The cache key
// is the device, the sample's problem count and its terms per problem
// (log2 buckets) and the mode.
extern "C" crp_status crp_autotune_batch(const crp_plan_desc *base, int32_t nprob,
                                         const crp_sparse *A, const crp_sparse *B,
                                         int32_t sample_probs, const char *cache_path,
                                         crp_plan_desc *best, double *best_terms_per_s,
                                         void *stream) {
    if (!base || !A || !B || !best || nprob <= 0) {
        set_last_error("crp_autotune_batch: bad argument");
        return CRP_EINVAL;
    }
    *best = *base;
    const int32_t ns = sample_probs > 0 && sample_probs < nprob ? sample_probs : nprob;
    std::vector<crp_sparse> SA, SB;
    for (int32_t x = 0; x < ns; ++x) {
        const int64_t q = (int64_t)x * nprob / ns;
        SA.push_back(A[q]);
        SB.push_back(B[q]);
    }
    // terms of the sample, from the host copies of the vector lengths
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t terms = 0;
    {
        unsigned long long *d_t = nullptr;
        if (cudaMalloc(&d_t, 8) != cudaSuccess) return CRP_ENOMEM;
        for (int32_t x = 0; x < ns; ++x) {
            unsigned long long t = 0;
            if (SA[x].n_major > 0) {
                launch_count_terms(SA[x].ptr, SB[x].ptr, SA[x].n_major, d_t, s);
                cudaMemcpyAsync(&t, d_t, 8, cudaMemcpyDeviceToHost, s);
                cudaStreamSynchronize(s);
            }
            terms += t;
        }
        cudaFree(d_t);
    }
    char key[320];
    {
        cudaDeviceProp prop;
        int dev = 0;
        cudaGetDevice(&dev);
        cudaGetDeviceProperties(&prop, dev);
        std::string name = prop.name;
        for (auto &c : name) if (c == ' ') c = '_';
        snprintf(key, sizeof key, "batch:%s:N%d:T%d:t%d:m%d", name.c_str(), ilog2u((uint64_t)ns),
                 ilog2u(terms + 1), ilog2u(terms / (uint64_t)ns + 1), base->mode);
    }
    if (cache_lookup(cache_path, key, best, best_terms_per_s)) return CRP_OK;
    const uint32_t Ps[] = {64, 256, 1024, 4096};
    const uint32_t tiles[] = {16, 32, 64, 128};
    double best_tps = -1.0;
    for (uint32_t P : Ps) {
        for (uint32_t t : tiles) {
            crp_plan_desc d = *base;
            d.P = P;
            d.tile_vectors = t;
            crp_batch *b = nullptr;
            if (crp_batch_create(&b, &d, ns, SA.data(), SB.data(), 0, stream) != CRP_OK) continue;
            double ms_best = 1e30;
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                double ms = 0;
                ok = crp_batch_run(b) == CRP_OK && crp_batch_sync(b, &ms, nullptr) == CRP_OK;
                if (ok && rep > 0 && ms > 0) ms_best = std::min(ms_best, ms);
            }
            crp_batch_destroy(b);
            if (!ok || ms_best >= 1e29) continue;
            const double tps = (double)terms / (ms_best * 1e-3);
            if (tps > best_tps) {
                best_tps = tps;
                *best = d;
            }
        }
    }
    // then the dense tier on the best (P, tile): hot blocks of 64, 128 or 255 items
    // per problem and side
    if (best_tps > 0) {
        const crp_plan_desc base_best = *best;
        for (uint32_t R : {64u, 128u, 255u}) {
            crp_plan_desc d = base_best;
            d.hot_items = R;
            crp_batch *b = nullptr;
            if (crp_batch_create(&b, &d, ns, SA.data(), SB.data(), 0, stream) != CRP_OK) continue;
            double ms_best = 1e30;
            bool ok = true;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                double ms = 0;
                ok = crp_batch_run(b) == CRP_OK && crp_batch_sync(b, &ms, nullptr) == CRP_OK;
                if (ok && rep > 0 && ms > 0) ms_best = std::min(ms_best, ms);
            }
            crp_batch_destroy(b);
            if (!ok || ms_best >= 1e29) continue;
            const double tps = (double)terms / (ms_best * 1e-3);
            if (tps > best_tps) {
                best_tps = tps;
                *best = d;
            }
        }
    }
    if (best_tps < 0) {
        set_last_error("crp_autotune_batch: no candidate configuration ran");
        return CRP_ECUDA;
    }
    if (best_terms_per_s) *best_terms_per_s = best_tps;
    cache_store(cache_path, key, *best, best_tps);
    return CRP_OK;
}
