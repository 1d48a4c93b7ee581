// An exact column-row product that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code running under an external memory
// manager that owns the whole device (a serving runtime with a preallocated
// arena), code inside a region where allocation is forbidden or would
// synchronise the device, or plug-ins whose host process forbids the CUDA
// allocator.  crp_outer_product_noalloc serves them: the partition tables it
// needs live in a file-scope static device array of fixed size, so the caller
// only provides the inputs and the output arrays.
//
// Limits: 2^20 table slots (16 MiB, held by every device that loads the
// library until the process exits) shared by at most 1024 partitions.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "crp_internal.cuh"

namespace crp {

constexpr uint64_t kNoallocSlots = 1ull << 20;
constexpr uint32_t kNoallocMaxP = 1024;
constexpr int kNoallocMaxDevices = 64;

// The static scratch: partition tables, their offsets and masks, the device
// counters and the output cursor.
struct NoallocScratch {
    Slot slots[kNoallocSlots];
    unsigned long long part_off[kNoallocMaxP];
    unsigned long long part_mask[kNoallocMaxP];
    unsigned int part_full[kNoallocMaxP];
    DevCounters dc;
    unsigned long long cursor;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

__global__ void k_noalloc_layout(NoallocScratch *sc, uint32_t P, unsigned long long cap) {
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        sc->part_off[p] = (unsigned long long)p * cap;
        sc->part_mask[p] = cap - 1ull;
        sc->part_full[p] = 0u;
    }
}

// Write every live slot to the caller's arrays (unordered).  cursor counts
// all live entries even past `capacity`, so the host learns the needed size.
__global__ void k_noalloc_emit(NoallocScratch *sc, uint64_t n_slots, int value_type,
                               int32_t *i_out, int32_t *j_out, double *w_out, int64_t capacity) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n_slots;
         x += (uint64_t)gridDim.x * blockDim.x) {
        const Slot s = sc->slots[x];
        if (s.key == kEmptyKey) continue;
        const unsigned long long at = atomicAdd(&sc->cursor, 1ull);
        if ((int64_t)at >= capacity) continue;
        i_out[at] = (int32_t)(s.key >> 32);
        j_out[at] = (int32_t)(uint32_t)s.key;
        w_out[at] = value_type == CRP_I32 ? (double)(unsigned int)s.val
                                          : __longlong_as_double((long long)s.val);
    }
}

// Device address of the static scratch.  A __device__ variable lives in the
// module loaded into one CUDA context, so its address is looked up (with
// cudaGetSymbolAddress, the device current) once per device and context: the
// cache holds the unique id of the context the address belongs to, and a
// call made in another context (after cudaDeviceReset, or in a context the
// caller created with the driver API) looks the address up again.
struct ScratchAddr {
    unsigned long long ctx_id;
    NoallocScratch *addr;
};
static ScratchAddr g_scratch_addr[kNoallocMaxDevices];
static std::mutex g_scratch_mu;

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Unique id of the calling thread's current context (driver API, reached
// through the runtime's entry-point query so the library needs no -lcuda).
static cudaError_t current_context_id(unsigned long long *id) {
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000,
                                                         cudaEnableDefault, &q0);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return cudaErrorSymbolNotFound;
        get_current = (CtxGetCurrentFn)f0;
        get_id = (CtxGetIdFn)f1;
    }
    void *ctx = nullptr;
    if (get_current(&ctx) != 0 || !ctx) return cudaErrorInvalidResourceHandle;
    if (get_id(ctx, id) != 0) return cudaErrorInvalidResourceHandle;
    return cudaSuccess;
}

static cudaError_t scratch_address(int dev, NoallocScratch **out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    ScratchAddr &c = g_scratch_addr[dev];
    unsigned long long id = 0;
    // no current context yet (a first call before any other CUDA work), or
    // another context than the cached address belongs to: look it up; the
    // lookup also makes the device's primary context current
    if (current_context_id(&id) != cudaSuccess || !c.addr || c.ctx_id != id) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        e = current_context_id(&id);
        if (e != cudaSuccess) return e;
        c.addr = (NoallocScratch *)p;
        c.ctx_id = id;
    }
    *out = c.addr;
    return cudaSuccess;
}

}  // namespace crp

using namespace crp;

static crp_status noalloc_fail(crp_status st, const std::string &m) {
    set_last_error(m);
    return st;
}

static uint64_t sm64(uint64_t &s) {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" crp_status crp_outer_product_noalloc(const crp_plan_desc *desc, const crp_sparse *A,
                                                const crp_sparse *B, int32_t *i_out,
                                                int32_t *j_out, double *w_out, int64_t capacity,
                                                int64_t *n_out, void *stream) {
    if (!desc || !A || !B || !n_out) return noalloc_fail(CRP_EINVAL, "null argument");
    *n_out = 0;
    const crp_plan_desc &d = *desc;
    if (d.P == 0 || (d.P & (d.P - 1)) || d.P > kNoallocMaxP)
        return noalloc_fail(CRP_EINVAL, "P must be a power of two <= 1024 here");
    if (d.n_rows <= 0 || d.n_cols <= 0 || A->n_minor != d.n_rows || B->n_minor != d.n_cols ||
        A->n_major != B->n_major || A->n_major < 0)
        return noalloc_fail(CRP_EINVAL, "shapes of A, B and desc disagree");
    if (d.value_type != CRP_I32 && d.value_type != CRP_F32_COMP)
        return noalloc_fail(CRP_EINVAL, "unknown value_type");
    if (d.value_type == CRP_I32 && (A->val || B->val))
        return noalloc_fail(CRP_EINVAL, "CRP_I32 counts {0,1} inputs: val must be NULL");
    if (d.mode != CRP_FULL && d.mode != CRP_UPPER) return noalloc_fail(CRP_EINVAL, "unknown mode");
    if (capacity < 0 || (capacity > 0 && (!i_out || !j_out || !w_out)))
        return noalloc_fail(CRP_EINVAL, "bad output arrays");
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev >= kNoallocMaxDevices)
        return noalloc_fail(CRP_ECUDA, "no usable CUDA device");
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    NoallocScratch *sc = nullptr;
    cudaError_t e = scratch_address(dev, &sc);
    if (e != cudaSuccess)
        return noalloc_fail(CRP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));

    const unsigned long long cap = kNoallocSlots / d.P;
    uint32_t logP = 0;
    while ((1u << logP) < d.P) ++logP;
    HashPair hp;
    uint64_t sa = d.seed_a, sb = d.seed_b;
    hp.ha.a = sm64(sa);
    hp.ha.b = sm64(sa);
    hp.hb.a = sm64(sb);
    hp.hb.b = sm64(sb);
    hp.ha.shift = hp.hb.shift = 64u - (logP > 0 ? logP : 1u);
    hp.ha.mask = hp.hb.mask = d.P - 1u;

#define NA_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess) return noalloc_fail(CRP_ECUDA, std::string(#call) + ": " +      \
                                                   cudaGetErrorString(_e));                    \
    } while (0)
    // clear what must start at zero: the tables, counters and cursor
    NA_CUDA(launch_fill_empty(sc->slots, kNoallocSlots, s));
    k_noalloc_layout<<<(d.P + 255) / 256, 256, 0, s>>>(sc, d.P, cap);
    NA_CUDA(cudaGetLastError());
    NA_CUDA(cudaMemsetAsync(&sc->dc, 0, sizeof(DevCounters), s));
    NA_CUDA(cudaMemsetAsync(&sc->cursor, 0, sizeof(unsigned long long), s));

    if (A->n_major > 0) {
        AccumulateArgs a;
        a.a_ptr = A->ptr;
        a.a_idx = A->idx;
        a.a_val = A->val;
        a.b_ptr = B->ptr;
        a.b_idx = B->idx;
        a.b_val = B->val;
        a.K = A->n_major;
        a.n_rows = d.n_rows;
        a.n_cols = d.n_cols;
        a.groups = 1;
        a.group_begin = 0;
        a.group_end = 1;
        a.tile = 64;
        a.n_tiles = (uint32_t)((A->n_major + 63) / 64);
        a.mode = d.mode;
        a.use_match = 1;
        a.debug_checks = 0;
        a.direct = 1;
        a.smem_slots = 4096;
        a.hp = hp;
        a.tv.slots = sc->slots;
        a.tv.part_off = sc->part_off;
        a.tv.part_mask = sc->part_mask;
        a.tv.part_full = sc->part_full;
        a.tv.spill = nullptr;
        a.tv.spill_cap = 0;     // a full partition is reported, nothing is kept aside
        a.tv.dc = &sc->dc;
        a.tv.value_type = d.value_type;
        a.tv.summary = 0;          // exact tables
        a.tv.has_reserved = 0;
        const int per_sm = accumulate_max_blocks_per_sm(d.value_type, 4096, true);
        if (per_sm <= 0) return noalloc_fail(CRP_ECUDA, "accumulate kernel cannot be resident");
        NA_CUDA(launch_accumulate(a, nullptr, per_sm * sms, s));
    }
    k_noalloc_emit<<<sms * 4, 256, 0, s>>>(sc, kNoallocSlots, d.value_type, i_out, j_out, w_out,
                                          capacity);
    NA_CUDA(cudaGetLastError());
    unsigned long long count = 0;
    unsigned int status = 0;
    NA_CUDA(cudaMemcpyAsync(&count, &sc->cursor, sizeof count, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaMemcpyAsync(&status, &sc->dc.status, sizeof status, cudaMemcpyDeviceToHost, s));
    NA_CUDA(cudaStreamSynchronize(s));
#undef NA_CUDA
    if (status & (kStatusTableFull | kStatusSpillFull))
        // updates that met a full partition were dropped, so the cursor
        // undercounts the product's entries: report no count at all
        return noalloc_fail(CRP_ETABLE_FULL,
                            "the product has more entries than a partition of the static table "
                            "holds (2^20 slots over P partitions)");
    if (status) return noalloc_fail(CRP_ECUDA, "device status " + std::to_string(status));
    *n_out = (int64_t)count;
    if ((int64_t)count > capacity)
        return noalloc_fail(CRP_EINVAL, "output capacity too small; *n_out holds the size needed");
    return CRP_OK;
}
