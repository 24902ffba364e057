// Handle management, memory pool, status strings and the small C-ABI calls.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include <algorithm>

#include "internal.cuh"

namespace argcsr {

std::atomic<uint64_t> g_launches{0};

static thread_local char t_last_error[256] = "";

argcsr_status record_cuda(cudaError_t err, const char *where) {
    snprintf(t_last_error, sizeof t_last_error, "%s: %s (%s)", where, cudaGetErrorName(err),
             cudaGetErrorString(err));
    return err == cudaErrorMemoryAllocation ? ARGCSR_ENOMEM : ARGCSR_ECUDA;
}

void set_error_message(const char *msg) { snprintf(t_last_error, sizeof t_last_error, "%s", msg); }

// One pool per device, created on first use.  Its release threshold is
// unbounded so that memory freed by one conversion is reused by the next
// without returning to the driver; argcsr_trim_pool() gives it back.
static std::mutex g_pool_mutex;
static cudaMemPool_t g_pools[64];
static bool g_pool_made[64];

static argcsr_status device_pool(cudaMemPool_t *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return ARGCSR_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pool_made[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) return record_cuda(e, "cudaMemPoolCreate");
        uint64_t threshold = UINT64_MAX;
        e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &threshold);
        if (e != cudaSuccess) return record_cuda(e, "cudaMemPoolSetAttribute");
        g_pool_made[dev] = true;
    }
    *out = g_pools[dev];
    return ARGCSR_OK;
}

// A caller's allocator (argcsr_set_allocator) replaces the pool for every
// device allocation while it is set.  g_live counts the allocations not yet
// freed, so the allocator cannot change under memory it has to free.
struct UserAllocator {
    argcsr_alloc_fn alloc = nullptr;
    argcsr_free_fn free = nullptr;
    void *ctx = nullptr;
};
static std::mutex g_alloc_mutex;
static UserAllocator g_user;
static int64_t g_live = 0;

argcsr_status pool_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) return ARGCSR_OK;
    // round up so every array starts 256-byte aligned and vector loads of
    // the last slots stay inside the allocation
    bytes = (bytes + 255) & ~size_t(255);
    std::unique_lock<std::mutex> lock(g_alloc_mutex);
    const UserAllocator u = g_user;
    if (u.alloc) {
        void *q = u.alloc(bytes, reinterpret_cast<argcsr_stream_t>(s), u.ctx);
        if (!q) {
            set_error_message("allocator callback returned NULL");
            return ARGCSR_ENOMEM;
        }
        if (reinterpret_cast<uintptr_t>(q) % 256) {
            u.free(q, reinterpret_cast<argcsr_stream_t>(s), u.ctx);
            set_error_message("allocator callback returned memory that is not 256-byte aligned");
            return ARGCSR_EINVAL;
        }
        *p = q;
        ++g_live;
        return ARGCSR_OK;
    }
    lock.unlock();
    cudaMemPool_t pool;
    argcsr_status st = device_pool(&pool);
    if (st != ARGCSR_OK) return st;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return record_cuda(e, "cudaMallocFromPoolAsync");
    }
    lock.lock();
    ++g_live;
    return ARGCSR_OK;
}

void pool_free(void *p, cudaStream_t s) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (g_user.free) g_user.free(p, reinterpret_cast<argcsr_stream_t>(s), g_user.ctx);
    else cudaFreeAsync(p, s);
    --g_live;
}

}  // namespace argcsr

using namespace argcsr;

extern "C" {

ARGCSR_API const char *argcsr_status_string(argcsr_status status) {
    switch (status) {
        case ARGCSR_OK: return "ARGCSR_OK";
        case ARGCSR_EINVAL: return "ARGCSR_EINVAL: invalid argument or malformed CSR input";
        case ARGCSR_ENOMEM: return "ARGCSR_ENOMEM: device allocation failed";
        case ARGCSR_ECUDA: return "ARGCSR_ECUDA: CUDA error";
        case ARGCSR_EOVERFLOW: return "ARGCSR_EOVERFLOW: more than 2^31-1 slots";
        case ARGCSR_ENOTSUP: return "ARGCSR_ENOTSUP: not supported";
    }
    return "unknown argcsr status";
}

ARGCSR_API const char *argcsr_last_error_message(void) { return t_last_error; }

ARGCSR_API uint64_t argcsr_launch_count(void) { return g_launches.load(); }

ARGCSR_API const char *argcsr_version(void) { return "argcsr 0.1 sm_103a"; }

ARGCSR_API argcsr_status argcsr_trim_pool(void) {
    cudaMemPool_t pool;
    argcsr_status st = device_pool(&pool);
    if (st != ARGCSR_OK) return st;
    cudaError_t e = cudaMemPoolTrimTo(pool, 0);
    return e == cudaSuccess ? ARGCSR_OK : record_cuda(e, "cudaMemPoolTrimTo");
}

ARGCSR_API argcsr_status argcsr_info(argcsr_t A, argcsr_info_t *out) {
    if (!A || !out) return ARGCSR_EINVAL;
    out->n_rows = A->n_rows;
    out->n_cols = A->n_cols;
    out->nnz = A->nnz;
    out->n_groups = A->n_groups;
    out->n_slots = A->n_slots;
    out->group_size = A->G;
    out->desired_chunk_size = A->D;
    out->vec_width = A->V;
    out->one_thread_per_row = A->one_per_row;
    out->reserved = 0;
    out->dtype = A->dtype;
    const int64_t sv = (int64_t)dtype_size(A->dtype), sx = (int64_t)vec_size(A->dtype);
    out->spmv_bytes = A->nnz * (sv + 4) + (int64_t)A->n_cols * sx + (int64_t)A->n_rows * sx +
                      4 * (int64_t)A->n_rows + 16 * A->n_groups;
    out->device_bytes = A->device_bytes;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_device_arrays(argcsr_t A, const int32_t **d_groupInfo,
                                              const int32_t **d_threadsMapping,
                                              const int32_t **d_columns, const void **d_values) {
    if (!A) return ARGCSR_EINVAL;
    if (d_groupInfo) *d_groupInfo = reinterpret_cast<const int32_t *>(A->d_groupInfo);
    if (d_threadsMapping) *d_threadsMapping = A->d_threadsMapping;
    if (d_columns) *d_columns = A->d_columns;
    if (d_values) *d_values = A->d_values;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_export(argcsr_t A, int32_t *h_groupInfo, int32_t *h_threadsMapping,
                                       int32_t *h_columns, void *h_values) {
    if (!A) return ARGCSR_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return record_cuda(e, "argcsr_export: synchronize");
    struct { void *dst; const void *src; size_t bytes; } copies[4] = {
        {h_groupInfo, A->d_groupInfo, (size_t)A->n_groups * 16},
        {h_threadsMapping, A->d_threadsMapping, (size_t)A->n_rows * 4},
        {h_columns, A->d_columns, (size_t)A->n_slots * 4},
        {h_values, A->d_values, (size_t)A->n_slots * dtype_size(A->dtype)},
    };
    for (auto &c : copies) {
        if (!c.dst || c.bytes == 0) continue;
        e = cudaMemcpy(c.dst, c.src, c.bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return record_cuda(e, "argcsr_export: copy");
    }
    // the device keeps the group records in execution order; the format's
    // order is by row (every record names its first row, and groups tile the
    // rows, so sorting by it restores the order of Section 3 exactly)
    if (h_groupInfo && A->execution_order && A->n_groups > 1) {
        struct Rec { int32_t v[4]; };
        Rec *r = reinterpret_cast<Rec *>(h_groupInfo);
        std::sort(r, r + A->n_groups, [](const Rec &a, const Rec &b) { return a.v[0] < b.v[0]; });
    }
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_destroy(argcsr_t A, argcsr_stream_t stream) {
    if (!A) return ARGCSR_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pool_free(A->d_groupInfo, s);
    pool_free(A->d_threadsMapping, s);
    pool_free(A->d_columns, s);
    pool_free(A->d_values, s);
    pool_free(A->d_longGroups, s);
    delete A;
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ARGCSR_OK : record_cuda(e, "argcsr_destroy");
}

ARGCSR_API argcsr_status argcsr_spmv(argcsr_t A, const void *d_x, void *d_y, argcsr_stream_t stream) {
    if (!A) return ARGCSR_EINVAL;
    if (A->n_rows == 0) return ARGCSR_OK;
    if (!d_y || (!d_x && A->n_cols > 0)) return ARGCSR_EINVAL;
    const size_t es = vec_size(A->dtype);
    const char *x0 = static_cast<const char *>(d_x), *x1 = x0 + (size_t)A->n_cols * es;
    const char *y0 = static_cast<const char *>(d_y), *y1 = y0 + (size_t)A->n_rows * es;
    if (d_x && x0 < y1 && y0 < x1) return ARGCSR_EINVAL;  // x and y overlap
    return launch_spmv(A, d_x, d_y, reinterpret_cast<cudaStream_t>(stream));
}

ARGCSR_API argcsr_status argcsr_probe_gather(argcsr_t A, const void *d_x, int32_t mode,
                                             argcsr_stream_t stream) {
    if (!A || mode < 0 || (mode & 3) == 3 || mode > 15) return ARGCSR_EINVAL;
    if (A->dtype != ARGCSR_F64 || (A->G != 32 && (mode >> 2) != 0)) {
        set_error_message("argcsr_probe_gather: f64 handles only; load instruction choices for G = 32 only");
        return ARGCSR_ENOTSUP;
    }
    if (A->n_rows == 0) return ARGCSR_OK;
    if (!d_x && A->n_cols > 0 && (mode & 3) != 2) return ARGCSR_EINVAL;
    return launch_probe_gather(A, d_x, mode, reinterpret_cast<cudaStream_t>(stream));
}

ARGCSR_API argcsr_status argcsr_set_allocator(argcsr_alloc_fn alloc, argcsr_free_fn free_fn, void *ctx) {
    if (!alloc != !free_fn) return ARGCSR_EINVAL;
    std::lock_guard<std::mutex> lock(g_alloc_mutex);
    if (g_live != 0) {
        set_error_message("argcsr_set_allocator: device memory from the current allocator is still held");
        return ARGCSR_EINVAL;
    }
    g_user = UserAllocator{alloc, free_fn, ctx};
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_spmv_axpby(argcsr_t A, double alpha, const void *d_x, double beta,
                                           void *d_y, argcsr_stream_t stream) {
    if (!A) return ARGCSR_EINVAL;
    if (A->n_rows == 0) return ARGCSR_OK;
    if (!d_y || (!d_x && A->n_cols > 0)) return ARGCSR_EINVAL;
    const size_t es = vec_size(A->dtype);
    const char *x0 = static_cast<const char *>(d_x), *x1 = x0 + (size_t)A->n_cols * es;
    const char *y0 = static_cast<const char *>(d_y), *y1 = y0 + (size_t)A->n_rows * es;
    if (d_x && x0 < y1 && y0 < x1) return ARGCSR_EINVAL;  // x and y overlap
    return launch_spmv_axpby(A, alpha, d_x, beta, d_y, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
