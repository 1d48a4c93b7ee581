// Measurement helper: the rate of random updates into a region of a given
// size (an L2-resident region vs an HBM-resident one).  It is the empirical
// side of the update roofline used for the exact tables (one random sector
// read-modify-write per update); it is not on the product path.
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "crp_internal.cuh"

namespace crp {

__device__ __forceinline__ uint64_t probe_mix(uint64_t x) {
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}

// mode 0: 32-bit atomic add (no return value) at a random word.
__global__ void k_probe_red(unsigned int *words, uint64_t mask, uint64_t n, uint64_t salt) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&words[probe_mix(x ^ salt) & mask], 1u);
}

// mode 1: the exact-table pattern on 16-byte slots: read the key, claim an
// empty slot with a CAS (linear probing), add to the count.
__global__ void k_probe_table(Slot *slots, uint64_t mask, uint64_t n_keys, uint64_t n,
                              uint64_t salt) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long key = probe_mix(x ^ salt) % n_keys;
        unsigned long long h = slot_mix(key) & mask;
        for (unsigned long long probe = 0; probe <= mask; ++probe) {
            Slot *s = slots + h;
            unsigned long long k = *(volatile unsigned long long *)&s->key;
            if (k == kEmptyKey) {
                k = atomicCAS(&s->key, kEmptyKey, key);
                if (k == kEmptyKey) k = key;
            }
            if (k == key) {
                atomicAdd((unsigned int *)&s->val, 1u);
                break;
            }
            h = (h + 1) & mask;
        }
    }
}

}  // namespace crp

using namespace crp;

extern "C" crp_status crp_probe_update_rate(uint64_t region_bytes, uint64_t n_updates, int mode,
                                            double *ms_out) {
    if (!ms_out || region_bytes < 4096 || (region_bytes & (region_bytes - 1)) || mode < 0 ||
        mode > 1)
        return CRP_EINVAL;
    void *buf = nullptr;
    if (cudaMalloc(&buf, region_bytes) != cudaSuccess) return CRP_ENOMEM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = sms * 8;
    crp_status st = CRP_OK;
    if (mode == 0) {
        cudaMemset(buf, 0, region_bytes);
        const uint64_t mask = region_bytes / 4 - 1;
        k_probe_red<<<grid, 512>>>((unsigned int *)buf, mask, n_updates / 4, 1);  // warm
        cudaEventRecord(e0);
        k_probe_red<<<grid, 512>>>((unsigned int *)buf, mask, n_updates, 2);
        cudaEventRecord(e1);
    } else {
        const uint64_t nslots = region_bytes / sizeof(Slot);
        launch_fill_empty((Slot *)buf, nslots, 0);
        const uint64_t mask = nslots - 1;
        const uint64_t n_keys = nslots / 2;
        k_probe_table<<<grid, 512>>>((Slot *)buf, mask, n_keys, n_updates / 4, 1);  // warm
        cudaEventRecord(e0);
        k_probe_table<<<grid, 512>>>((Slot *)buf, mask, n_keys, n_updates, 2);
        cudaEventRecord(e1);
    }
    if (cudaEventSynchronize(e1) != cudaSuccess) st = CRP_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    *ms_out = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    return st;
}
