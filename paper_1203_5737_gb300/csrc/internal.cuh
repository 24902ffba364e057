// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <atomic>

#include "argcsr.h"

namespace argcsr {

// Bits of the device-side validation word written by the conversion kernels.
enum : unsigned {
    kBadRowPointers = 1u,  // rowPointers[0] != 0, decreasing, or last != nnz
    kBadColumn      = 2u,  // a column outside [0, n_cols)
    kSlotOverflow   = 4u,  // more than 2^31 - 1 slots
};

// Programmatic dependent launch.  A kernel launched with the programmatic
// stream serialization attribute (launch_pdl) may start while the kernel
// ahead of it on the stream is still running; pdl_wait() returns once that
// kernel has completed and its writes are visible, so nothing it writes may
// be touched before the call.  pdl_trigger() lets the next such kernel
// launch.  For kernels launched without the attribute both return at once.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr = {};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Totals produced on the device during conversion and read back once.
struct DeviceTotals {
    unsigned status;
    unsigned pad;
    long long n_groups;
    long long n_slots;
    long long n_long;   // groups with more than kLongChunk slot rows
};

// A G = 32 group whose chunk size exceeds this is a "long group": its slot
// rows are shared out among the 8 warps of one of the first blocks of the
// product kernels rather than walked by one warp.  k_fill lists them.
constexpr int kLongChunk = 64;

}  // namespace argcsr

struct argcsr_matrix {
    int device;
    int32_t n_rows, n_cols;
    int64_t nnz;
    int32_t G, D, V;
    int32_t one_per_row;        // 1: every row one thread (no adaptive step)
    argcsr_dtype dtype;
    int64_t n_groups, n_slots;
    int4 *d_groupInfo;          // {firstRow, size, offset, chunkSize}, in execution order
                                // (execution_order: by chunk size, largest first) or row order
    int32_t *d_threadsMapping;  // group-local inclusive prefix of threads per row
    int32_t *d_columns;         // S slots, -1 = padding
    void *d_values;             // S slots of dtype, +0.0 = padding
    int64_t device_bytes;
    int32_t *d_longGroups = nullptr;   // positions in d_groupInfo of the long groups (G 32, V 1)
    int64_t n_long = 0;
    int32_t execution_order = 0;       // d_groupInfo records sorted by chunk size, not by row
};

namespace argcsr {

extern std::atomic<uint64_t> g_launches;

inline void count_launches(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// Tracing: while argcsr_trace_begin() is in effect, a TraceScope records an
// event pair around the launches made during its lifetime.
int trace_start(const char *name, cudaStream_t s);
bool trace_active();
void trace_stop(int token, cudaStream_t s);
struct TraceScope {
    int token;
    cudaStream_t s;
    TraceScope(const char *name, cudaStream_t stream) : token(trace_start(name, stream)), s(stream) {}
    ~TraceScope() { trace_stop(token, s); }
};

// Record a CUDA error for argcsr_last_error_message(); returns ARGCSR_ECUDA
// (or ARGCSR_ENOMEM for allocation failures).
argcsr_status record_cuda(cudaError_t err, const char *where);
// Set the text returned by argcsr_last_error_message() for a non-CUDA error.
void set_error_message(const char *msg);

// Stream-ordered allocation from the library's per-device pool.
argcsr_status pool_alloc(void **p, size_t bytes, cudaStream_t s);
void pool_free(void *p, cudaStream_t s);

inline size_t dtype_size(argcsr_dtype t) {
    return t == ARGCSR_F64 ? 8 : t == ARGCSR_F32 ? 4 : 2;
}
inline size_t vec_size(argcsr_dtype t) {  // element size of x and y
    return t == ARGCSR_F64 ? 8 : 4;
}

// Defined in spmv.cu: launch the ARG-CSR SpMV kernel for a handle.
argcsr_status launch_probe_gather(const argcsr_matrix *A, const void *x, int mode, cudaStream_t s);
argcsr_status launch_spmv(const argcsr_matrix *A, const void *x, void *y, cudaStream_t s);
// One matrix of a batch (spmm.cu builds the array on the device).
struct BatchDesc {
    const int4 *gi;
    const int *tm;
    const int *cols;
    const void *vals;
    long long rowBase;   // first row of this matrix in the packed Y
    long long colBase;   // first row of this matrix in the packed X
    long long nGroups;   // groups of this matrix
    int nCols;           // columns of this matrix
    int reserved;
};
// y = A x for every matrix of a batch (k = 1, G = 32, V = 1): one block per
// matrix in `order`, x staged in shared memory when it fits (spmv.cu).
argcsr_status prepare_batch_spmv();
argcsr_status launch_batch_spmv(const BatchDesc *desc, const int *order, int count, int maxCols,
                                long long totalGroups, argcsr_dtype dtype, const void *X, void *Y,
                                cudaStream_t s);
// y = alpha A x + beta y (y not read when beta is 0).
argcsr_status launch_spmv_axpby(const argcsr_matrix *A, double alpha, const void *x, double beta,
                                void *y, cudaStream_t s);
// Plain CSR FP64 (vector kernel): y = A x and r = b - A x.
argcsr_status launch_csr_vector_f64(int32_t n, int32_t n_cols, int64_t nnz, const int32_t *rp,
                                    const int32_t *cols, const double *vals, const double *x,
                                    double *y, cudaStream_t s);
argcsr_status launch_csr_residual_f64(int32_t n, int32_t n_cols, int64_t nnz, const int32_t *rp,
                                      const int32_t *cols, const double *vals, const double *b,
                                      const double *x, double *r, cudaStream_t s);
// r = b - A x with FP64 vectors and FP64 accumulation, for any storage type
// (stored values are widened exactly).
argcsr_status launch_residual_f64(const argcsr_matrix *A, const double *b, const double *x,
                                  double *r, cudaStream_t s);

// A conjugate-gradient solve as a resumable job (solver.cu): start() and
// advance() enqueue work on the job's stream and return at once; a step is
// complete when step_done() (or wait_step() returns).
class CgJob {
public:
    virtual ~CgJob() = default;
    virtual argcsr_status start() = 0;
    virtual argcsr_status advance() = 0;
    virtual bool step_done() const = 0;
    virtual argcsr_status wait_step() = 0;
    virtual bool finished() const = 0;
    virtual argcsr_status status() const = 0;
    virtual void result(argcsr_cg_result *r) const = 0;
    virtual size_t workspace_bytes() const = 0;
};
CgJob *make_cg_job(const argcsr_matrix *A, const argcsr_matrix *Ares, const double *b, double *x,
                   const argcsr_cg_params &P, cudaStream_t s);
size_t cg_job_bytes(const argcsr_matrix *A);

// SpMM launch (spmm.cu), for the serving engine.
argcsr_status launch_spmm_public(const argcsr_matrix *A, int k, const void *X, long long ldx, void *Y,
                                 long long ldy, cudaStream_t s);

}  // namespace argcsr

#define ARGCSR_CHECK_LAUNCH(where)                                   \
    do {                                                             \
        cudaError_t e_ = cudaGetLastError();                         \
        if (e_ != cudaSuccess) return argcsr::record_cuda(e_, where); \
    } while (0)
