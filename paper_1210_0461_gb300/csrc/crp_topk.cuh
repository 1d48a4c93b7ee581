// Top-k certified from the hot block ({0,1} inputs, exact tables): the
// kernels of crp_topk.cu that crp_topk runs before any table scan.
#pragma once

#include "crp_internal.cuh"

namespace crp {

cudaError_t launch_degrees(const int32_t *idx, int64_t nnz, int32_t n, const uint16_t *rank,
                           uint32_t R, const int64_t *items, unsigned long long *deg,
                           int sm_count, cudaStream_t s);
cudaError_t launch_max_outside(const unsigned long long *deg, int32_t n, const uint16_t *rank,
                               uint32_t R, unsigned long long *out, cudaStream_t s);
cudaError_t launch_topk_hot_candidates(const Slot *slots, const unsigned long long *part_off,
                                       const unsigned long long *part_mask, const HashPair &hp,
                                       const int64_t *items_a, const int64_t *items_b, uint32_t R,
                                       int upper_only, TopkCand *out, unsigned int *count,
                                       cudaStream_t s);

}  // namespace crp
