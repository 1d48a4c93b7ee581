// Count-Sketch estimates (Preliminaries, "Count-Sketch"): the estimate of
// entry e from one sketch is s(e) CS[h(e)]; from t independent sketches it is
// the median of the t estimates.  One thread per queried entry; the t
// estimates sit in a small local array sorted by insertion.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "crp_internal.cuh"

namespace crp {

__global__ void k_sketch_estimate(SketchSet S, const int32_t *__restrict__ qi,
                                  const int32_t *__restrict__ qj, int64_t n, int32_t n_rows,
                                  int32_t n_cols, double *__restrict__ out, unsigned int *bad) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = qi[q], b = qj[q];
        if (a < 0 || a >= n_rows || b < 0 || b >= n_cols) {
            atomicOr(bad, 1u);
            out[q] = nan("");
            continue;
        }
        double v[kSketchMaxT];
        for (int r = 0; r < S.t; ++r) {
            const uint32_t p = partition_hash(S.hp[r], (uint32_t)a, (uint32_t)b);
            const double x = S.value_type == CRP_I32
                                 ? (double)((const long long *)S.cs[r])[p]
                                 : ((const double *)S.cs[r])[p];
            double e = sign_negative(S.sg[r], (uint32_t)a, (uint32_t)b) ? -x : x;
            int m = r;   // insertion into v[0..r)
            while (m > 0 && v[m - 1] > e) {
                v[m] = v[m - 1];
                --m;
            }
            v[m] = e;
        }
        const int h = S.t >> 1;
        out[q] = (S.t & 1) ? v[h] : 0.5 * (v[h - 1] + v[h]);
    }
}

cudaError_t launch_sketch_estimate(const SketchSet &S, const int32_t *i, const int32_t *j,
                                   int64_t n, int32_t n_rows, int32_t n_cols, double *out,
                                   unsigned int *bad, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t want = (n + threads - 1) / threads;
    const int grid = (int)(want < 4096 ? want : 4096);
    k_sketch_estimate<<<grid, threads, 0, s>>>(S, i, j, n, n_rows, n_cols, out, bad);
    return cudaGetLastError();
}

}  // namespace crp
