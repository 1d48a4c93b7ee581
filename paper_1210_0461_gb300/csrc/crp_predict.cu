// Predicting heavy pairs from a prefix of the stream, and reserving exact
// counters for them (summary mode).  Not in the paper.
//
//  1. item counts c_i over a prefix of the transactions (the marginals);
//  2. the R items of largest prefix count;
//  3. candidate pairs i < j among them, with features
//     (log(1 + c_i), log(1 + c_j)) / log(1 + max c);
//  4. a score per candidate: the trained network (crp_mlp_forward), or the
//     product-of-marginals heuristic log(1 + c_i) + log(1 + c_j);
//  5. the n candidates of highest score -> crp_reserve.
// Selections are MSD radix selects on order-preserving 32-bit keys (8-bit
// digits); ties at the threshold are taken in arbitrary order.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "crp_internal.cuh"

extern "C" crp_status crp_mlp_forward(const float *params, const float *x, float *y, int64_t n,
                                      void *stream);
extern "C" crp_status crp_reserve(crp_plan *plan, const uint64_t *keys, int32_t n);

namespace crp {

// Order-preserving key of a float (larger float -> larger key).
__global__ void k_float_keys(const float *v, int64_t n, uint32_t *key) {
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = __float_as_uint(v[x]);
        key[x] = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    }
}

__global__ void k_max_u32(const unsigned int *v, int64_t n, unsigned int *mx) {
    unsigned int m = 0;
    for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x)
        m = max(m, v[x]);
    atomicMax(mx, m);
}

// Candidate pairs: slot a * R + b for a < b holds (min, max) of the two items.
__global__ void k_candidates(const int64_t *items, int32_t R, const unsigned int *cnt,
                             const unsigned int *mx, int32_t *ci, int32_t *cj, float *x) {
    const float scale = logf(1.0f + (float)*mx);
    const float inv = scale > 0.f ? 1.0f / scale : 0.f;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < (int64_t)R * R;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = (int32_t)(s / R), b = (int32_t)(s % R);
        if (b <= a) continue;
        const int32_t ia = (int32_t)items[a], ib = (int32_t)items[b];
        const int32_t i = ia < ib ? ia : ib, j = ia < ib ? ib : ia;
        const int64_t o = (int64_t)a * (2 * R - a - 1) / 2 + (b - a - 1);
        ci[o] = i;
        cj[o] = j;
        x[2 * o] = logf(1.0f + (float)cnt[i]) * inv;
        x[2 * o + 1] = logf(1.0f + (float)cnt[j]) * inv;
    }
}

__global__ void k_heuristic(const float *x, int64_t n, float *score) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x)
        score[s] = x[2 * s] + x[2 * s + 1];
}

__global__ void k_pair_keys(const int64_t *sel, int64_t n, const int32_t *ci, const int32_t *cj,
                            int full, unsigned long long *keys) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = sel[s];
        const uint32_t i = (uint32_t)ci[c], j = (uint32_t)cj[c];
        keys[s] = ((unsigned long long)i << 32) | j;
        if (full) keys[n + s] = ((unsigned long long)j << 32) | i;
    }
}

}  // namespace crp

using namespace crp;

struct CandBufs {
    unsigned int *cnt = nullptr, *mx = nullptr, *scratch = nullptr;
    uint32_t *keys = nullptr;
    int64_t *items = nullptr;
};

extern "C" crp_status crp_candidate_pairs(const crp_sparse *prefix, int32_t n_items, int32_t R,
                                          int32_t *i_out, int32_t *j_out, float *x_out,
                                          int64_t capacity, int64_t *n_out, void *stream) {
    if (!prefix || !n_out || n_items <= 0 || R < 2 || R > n_items) {
        set_last_error("crp_candidate_pairs: bad argument");
        return CRP_EINVAL;
    }
    const int64_t nc = (int64_t)R * (R - 1) / 2;
    *n_out = nc;
    if (capacity < nc || !i_out || !j_out || !x_out) {
        set_last_error("crp_candidate_pairs: capacity below R(R-1)/2");
        return CRP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    CandBufs b;
    crp_status st = CRP_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == CRP_OK) {
            set_last_error(std::string("crp_candidate_pairs: ") + cudaGetErrorString(e));
            st = e == cudaErrorMemoryAllocation ? CRP_ENOMEM : CRP_ECUDA;
        }
        return st == CRP_OK;
    };
    if (ok(cudaMalloc(&b.cnt, (size_t)n_items * 4)) && ok(cudaMalloc(&b.mx, 4)) &&
        ok(cudaMalloc(&b.scratch, 260 * 4)) && ok(cudaMalloc(&b.items, (size_t)R * 8))) {
        ok(cudaMemsetAsync(b.cnt, 0, (size_t)n_items * 4, s));
        ok(cudaMemsetAsync(b.mx, 0, 4, s));
        ok(launch_item_counts(prefix->idx, prefix->nnz, n_items, b.cnt, s));
        k_max_u32<<<select_grid_for(n_items), 256, 0, s>>>(b.cnt, n_items, b.mx);
        ok(cudaGetLastError());
        if (st == CRP_OK) ok(select_top(b.cnt, n_items, R, b.items, b.scratch, s));
        if (st == CRP_OK) {
            k_candidates<<<select_grid_for((int64_t)R * R), 256, 0, s>>>(b.items, R, b.cnt, b.mx, i_out,
                                                                  j_out, x_out);
            ok(cudaGetLastError());
            ok(cudaStreamSynchronize(s));
        }
    }
    cudaFree(b.cnt);
    cudaFree(b.mx);
    cudaFree(b.scratch);
    cudaFree(b.items);
    return st;
}

extern "C" crp_status crp_predict_reserve(crp_plan *plan, const crp_sparse *prefix, int32_t n_items,
                                          const float *params, int32_t R, int32_t n_reserve,
                                          int32_t full_mode, void *stream) {
    if (!plan || !prefix || R < 2 || n_reserve <= 0) {
        set_last_error("crp_predict_reserve: bad argument");
        return CRP_EINVAL;
    }
    const int64_t nc = (int64_t)R * (R - 1) / 2;
    const int64_t take = n_reserve < nc ? n_reserve : nc;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *ci = nullptr, *cj = nullptr;
    float *x = nullptr, *score = nullptr;
    uint32_t *key = nullptr;
    int64_t *sel = nullptr;
    unsigned long long *keys = nullptr;
    unsigned int *scratch = nullptr;
    crp_status st = CRP_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && st == CRP_OK) {
            set_last_error(std::string("crp_predict_reserve: ") + cudaGetErrorString(e));
            st = e == cudaErrorMemoryAllocation ? CRP_ENOMEM : CRP_ECUDA;
        }
        return st == CRP_OK;
    };
    if (ok(cudaMalloc(&ci, nc * 4)) && ok(cudaMalloc(&cj, nc * 4)) && ok(cudaMalloc(&x, nc * 8)) &&
        ok(cudaMalloc(&score, nc * 4)) && ok(cudaMalloc(&key, nc * 4)) &&
        ok(cudaMalloc(&sel, take * 8)) && ok(cudaMalloc(&keys, take * 16)) &&
        ok(cudaMalloc(&scratch, 260 * 4))) {
        int64_t n = 0;
        st = crp_candidate_pairs(prefix, n_items, R, ci, cj, x, nc, &n, stream);
        if (st == CRP_OK) {
            if (params) st = crp_mlp_forward(params, x, score, nc, stream);
            else {
                k_heuristic<<<select_grid_for(nc), 256, 0, s>>>(x, nc, score);
                ok(cudaGetLastError());
            }
        }
        if (st == CRP_OK) {
            k_float_keys<<<select_grid_for(nc), 256, 0, s>>>(score, nc, key);
            ok(cudaGetLastError());
        }
        if (st == CRP_OK) ok(select_top(key, nc, take, sel, scratch, s));
        if (st == CRP_OK) {
            k_pair_keys<<<select_grid_for(take), 256, 0, s>>>(sel, take, ci, cj, full_mode ? 1 : 0, keys);
            ok(cudaGetLastError());
            ok(cudaStreamSynchronize(s));
        }
        if (st == CRP_OK)
            st = crp_reserve(plan, (const uint64_t *)keys, (int32_t)(full_mode ? 2 * take : take));
    }
    cudaFree(ci);
    cudaFree(cj);
    cudaFree(x);
    cudaFree(score);
    cudaFree(key);
    cudaFree(sel);
    cudaFree(keys);
    cudaFree(scratch);
    return st;
}
