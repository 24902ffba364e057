// Conjugate gradients on ARG-CSR, with FP64 iterative refinement around a
// low-precision inner solve.  This is the iterative-solver use of SpMV that
// motivates the format (Section 1 of Heller & Oberhuber: SpMV "is a key part
// of many iterative solvers"); the solver itself is textbook CG.
//
// Refinement (outer loop, FP64 on the device):
//     r = b - A x        (FP64 vectors, FP64 accumulation; stored values of
//                         any type are widened exactly)
//     stop when ||r|| <= tol ||b||
//     solve A d = r / ||r|| approximately with CG in the working type WT
//     x += ||r|| d       (FP64)
// The inner CG runs in WT = float for FP32/BF16 storage (FP32 accumulation)
// and in WT = double for FP64 storage.  Every scalar of the iteration (rho,
// alpha, beta, norms) stays on the device: each reduction kernel writes one
// partial per block and the last block to finish adds the partials in a
// fixed order, so results do not depend on scheduling and no host read is
// needed inside an iteration.  The host reads rho every `check_every` inner
// iterations to decide convergence.
#include <math.h>

#include <mutex>
#include <new>
#include <vector>

#include "internal.cuh"

namespace argcsr {
namespace {

constexpr int kVecBlocks = 152 * 8;  // largest grid of the vector kernels (= partials)
constexpr int kUnroll = 16;          // independent elements per thread per step
constexpr int kVecThreads = 256;

// Grid of the vector kernels for n elements: one block per kUnroll * 256
// elements, at most kVecBlocks.  Small solves then occupy few SMs, so that
// the serving engine's concurrent jobs really run side by side.
inline int vec_blocks(long long n) {
    const long long b = (n + (long long)kUnroll * kVecThreads - 1) / ((long long)kUnroll * kVecThreads);
    return (int)(b < 1 ? 1 : b > kVecBlocks ? kVecBlocks : b);
}

// Device-resident scalars of a solve.
struct CgState {
    double rho;        // r.r of the inner iteration
    double rho0;       // r.r at the start of the inner solve
    double alpha, beta;
    double norm2;      // ||r||^2 of the FP64 residual
    double bnorm2;     // ||b||^2
    unsigned counter;  // blocks finished in the current reduction
    unsigned pad;
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block (valid in thread 0).
template <typename T>
__device__ __forceinline__ T block_sum(T v) {
    __shared__ T sh[kVecThreads / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    T t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kVecThreads / 32 ? sh[threadIdx.x] : T(0);
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Every block contributes `partial`; returns true in thread 0 of the last
// block to finish, with the sum of all partials (in block order) in *total.
// Within a block the sum is taken in the partial's own type (FP32 for the
// FP32 inner solve: on GB300 an FP64 add costs 32 times an FP32 one), across
// blocks in FP64.
template <typename T>
__device__ bool last_block_total(T partial, double *partials, unsigned *counter, double *total) {
    __shared__ bool s_last;
    const double bsum = (double)block_sum<T>(partial);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bsum;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return false;
    __threadfence();
    double t = 0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) t += ((volatile double *)partials)[i];
    t = block_sum<double>(t);
    if (threadIdx.x == 0) {
        *total = t;
        *counter = 0;  // ready for the next reduction
    }
    return threadIdx.x == 0;
}

// Grid-stride loop over [0, n), kUnroll independent elements per thread and
// step so that several loads are in flight: BODY(i) runs for each element.
#define FOR_EACH_ELEMENT(n, BODY)                                                         \
    do {                                                                                  \
        const long long stride_ = (long long)gridDim.x * blockDim.x;                      \
        for (long long i0_ = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0_ < (n); \
             i0_ += kUnroll * stride_) {                                                  \
            _Pragma("unroll") for (int u_ = 0; u_ < kUnroll; ++u_) {                      \
                const long long i = i0_ + u_ * stride_;                                   \
                if (i < (n)) { BODY; }                                                    \
            }                                                                             \
        }                                                                                 \
    } while (0)

// The FP32 inner iteration's vectors in 16-byte pieces of 4 floats: a quarter
// of the load instructions and L1 requests of element loads for the same
// bytes (the solver allocates the vectors, 256-byte aligned).  The FP64
// iteration keeps element loads: with pieces of 2 doubles the kernels need
// twice the registers and were 12 % slower.
template <typename WT>
__device__ __forceinline__ void ld16(const WT *__restrict__ p, long long iv, WT (&out)[16 / sizeof(WT)]) {
    const uint4 u = reinterpret_cast<const uint4 *>(p)[iv];
    memcpy(out, &u, 16);
}
template <typename WT>
__device__ __forceinline__ void st16(WT *__restrict__ p, long long iv, const WT (&in)[16 / sizeof(WT)]) {
    uint4 u;
    memcpy(&u, in, 16);
    reinterpret_cast<uint4 *>(p)[iv] = u;
}

// Grid-stride loop over the n / W whole 16-byte pieces of [0, n), kUnroll / W
// pieces per thread and step (the same kUnroll elements as
// FOR_EACH_ELEMENT): fv(iv) for each piece, then fs(i) for the elements
// after the last whole piece.
template <int W, typename FV, typename FS>
__device__ __forceinline__ void for_each_piece(long long n, FV &&fv, FS &&fs) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nv = n / W;
    for (long long v0 = t; v0 < nv; v0 += (kUnroll / W) * stride) {
#pragma unroll
        for (int u = 0; u < kUnroll / W; ++u) {
            const long long iv = v0 + u * stride;
            if (iv < nv) fv(iv);
        }
    }
    for (long long i = nv * W + t; i < n; i += stride) fs(i);
}

template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_cg_alpha(const WT *__restrict__ p, const WT *__restrict__ q, long long n, double *partials,
           CgState *S) {
    constexpr int W = 16 / sizeof(WT);
    WT acc = 0;
    if constexpr (W == 4) {
        for_each_piece<W>(n, [&](long long iv) {
            WT a[W], b[W];
            ld16(p, iv, a);
            ld16(q, iv, b);
#pragma unroll
            for (int k = 0; k < W; ++k) acc = fma(a[k], b[k], acc);
        }, [&](long long i) { acc = fma(p[i], q[i], acc); });
    } else {
        FOR_EACH_ELEMENT(n, acc = fma(p[i], q[i], acc));
    }
    double pq;
    if (last_block_total<WT>(acc, partials, &S->counter, &pq))
        S->alpha = pq != 0.0 ? S->rho / pq : 0.0;
}

// x += alpha p; r -= alpha q; then rho_new = r.r, beta = rho_new / rho.
template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_cg_update(WT *__restrict__ x, WT *__restrict__ r, const WT *__restrict__ p,
            const WT *__restrict__ q, long long n, double *partials, CgState *S) {
    constexpr int W = 16 / sizeof(WT);
    const WT alpha = (WT)S->alpha;
    WT acc = 0;
    auto one = [&](long long i) {
        x[i] = fma(alpha, p[i], x[i]);
        const WT ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    };
    if constexpr (W == 4) {
        for_each_piece<W>(n, [&](long long iv) {
            WT xv[W], pv[W], qv[W], rv[W];
            ld16(x, iv, xv);
            ld16(p, iv, pv);
            ld16(q, iv, qv);
            ld16(r, iv, rv);
#pragma unroll
            for (int k = 0; k < W; ++k) {
                xv[k] = fma(alpha, pv[k], xv[k]);
                rv[k] = fma(-alpha, qv[k], rv[k]);
                acc = fma(rv[k], rv[k], acc);
            }
            st16(x, iv, xv);
            st16(r, iv, rv);
        }, one);
    } else {
        FOR_EACH_ELEMENT(n, one(i));
    }
    double rho_new;
    if (last_block_total<WT>(acc, partials, &S->counter, &rho_new)) {
        S->beta = S->rho != 0.0 ? rho_new / S->rho : 0.0;
        S->rho = rho_new;
    }
}

template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_cg_direction(WT *__restrict__ p, const WT *__restrict__ r, long long n, const CgState *S) {
    constexpr int W = 16 / sizeof(WT);
    const WT beta = (WT)S->beta;
    if constexpr (W == 4) {
        for_each_piece<W>(n, [&](long long iv) {
            WT pv[W], rv[W];
            ld16(p, iv, pv);
            ld16(r, iv, rv);
#pragma unroll
            for (int k = 0; k < W; ++k) pv[k] = fma(beta, pv[k], rv[k]);
            st16(p, iv, pv);
        }, [&](long long i) { p[i] = fma(beta, p[i], r[i]); });
    } else {
        FOR_EACH_ELEMENT(n, p[i] = fma(beta, p[i], r[i]));
    }
}

// ||v||^2 in FP64 into *out (norm2 or bnorm2 of the state).
__global__ void __launch_bounds__(kVecThreads)
k_norm2_f64(const double *__restrict__ v, long long n, double *partials, CgState *S, int which) {
    double acc = 0;
    FOR_EACH_ELEMENT(n, acc = fma(v[i], v[i], acc));
    double t;
    if (last_block_total<double>(acc, partials, &S->counter, &t)) {
        if (which == 0) S->norm2 = t; else S->bnorm2 = t;
    }
}

// Start an inner solve: r = r64 / ||r64||, p = r, d = 0, rho = rho0 = r.r.
template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_ir_start(const double *__restrict__ r64, WT *__restrict__ r, WT *__restrict__ p,
           WT *__restrict__ d, long long n, double *partials, CgState *S) {
    const double scale = S->norm2 > 0.0 ? 1.0 / sqrt(S->norm2) : 0.0;
    WT acc = 0;
    FOR_EACH_ELEMENT(n, {
        const WT ri = (WT)(r64[i] * scale);
        r[i] = ri;
        p[i] = ri;
        d[i] = 0;
        acc = fma(ri, ri, acc);
    });
    double t;
    if (last_block_total<WT>(acc, partials, &S->counter, &t)) {
        S->rho = t;
        S->rho0 = t;
    }
}

// x += ||r64|| d (FP64).
template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_ir_correct(double *__restrict__ x, const WT *__restrict__ d, long long n, const CgState *S) {
    const double scale = sqrt(S->norm2);
    FOR_EACH_ELEMENT(n, x[i] = fma(scale, (double)d[i], x[i]));
}

// The matrix operator used by the solver: ARG-CSR or plain CSR.
struct Operator {
    const argcsr_matrix *A = nullptr;        // ARG-CSR (inner products)
    const argcsr_matrix *Ares = nullptr;     // ARG-CSR (FP64 residual)
    // plain CSR FP64 (baseline)
    int32_t n = 0, n_cols = 0;
    int64_t nnz = 0;
    const int32_t *rp = nullptr, *cols = nullptr;
    const double *vals = nullptr;

    argcsr_status apply(const void *x, void *y, cudaStream_t s) const {
        if (A) return launch_spmv(A, x, y, s);
        return launch_csr_vector_f64(n, n_cols, nnz, rp, cols, vals, static_cast<const double *>(x),
                                     static_cast<double *>(y), s);
    }
    argcsr_status residual(const double *b, const double *x, double *r, cudaStream_t s) const {
        if (Ares) return launch_residual_f64(Ares, b, x, r, s);
        return launch_csr_residual_f64(n, n_cols, nnz, rp, cols, vals, b, x, r, s);
    }
};

// Pinned host copies of the solver state, reused across solves.
std::mutex g_pinned_mu;
std::vector<CgState *> g_pinned_free;

CgState *take_pinned() {
    {
        std::lock_guard<std::mutex> lock(g_pinned_mu);
        if (!g_pinned_free.empty()) {
            CgState *p = g_pinned_free.back();
            g_pinned_free.pop_back();
            return p;
        }
    }
    CgState *p = nullptr;
    if (cudaHostAlloc((void **)&p, sizeof(CgState), cudaHostAllocDefault) != cudaSuccess) return nullptr;
    return p;
}

void give_pinned(CgState *p) {
    if (!p) return;
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    g_pinned_free.push_back(p);
}

// One solve as a resumable state machine: every call to advance() enqueues
// the next block of work on the job's stream (ending with an asynchronous
// copy of the device state to pinned host memory and an event) and returns
// at once; when the event has completed, the next advance() reads the copy
// and decides.  A synchronous solve loops on the event; the serving engine
// interleaves many jobs on their own streams.
template <typename WT>
class CgJobT final : public CgJob {
public:
    CgJobT(const Operator &op, long long n, const double *b, double *x, const argcsr_cg_params &P,
           cudaStream_t s)
        : op_(op), n_(n), b_(b), x_(x), P_(P), s_(s), blocks_(vec_blocks(n)) {}

    ~CgJobT() override {
        pool_free(r_, s_); pool_free(p_, s_); pool_free(q_, s_); pool_free(d_, s_);
        pool_free(r64_, s_); pool_free(partials_, s_); pool_free(S_, s_);
        if (ev_) cudaEventDestroy(ev_);
        if (inner_exec_) cudaGraphExecDestroy(inner_exec_);
        give_pinned(hS_);
    }

    size_t workspace_bytes() const override { return bytes_for(n_); }
    static size_t bytes_for(long long n) {
        return 4 * (size_t)n * sizeof(WT) + (size_t)n * 8 + (size_t)kVecBlocks * 8 + sizeof(CgState) + 7 * 256;
    }

    argcsr_status start() override {
        const size_t vb = (size_t)n_ * sizeof(WT);
        argcsr_status st;
        if ((st = pool_alloc((void **)&r_, vb, s_)) || (st = pool_alloc((void **)&p_, vb, s_)) ||
            (st = pool_alloc((void **)&q_, vb, s_)) || (st = pool_alloc((void **)&d_, vb, s_)) ||
            (st = pool_alloc((void **)&r64_, (size_t)n_ * 8, s_)) ||
            (st = pool_alloc((void **)&partials_, (size_t)kVecBlocks * 8, s_)) ||
            (st = pool_alloc((void **)&S_, sizeof(CgState), s_)))
            return fail(st);
        hS_ = take_pinned();
        if (!hS_) return fail(ARGCSR_ENOMEM);
        cudaError_t e = cudaEventCreateWithFlags(&ev_, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMemsetAsync(S_, 0, sizeof(CgState), s_);
        if (e != cudaSuccess) return fail(record_cuda(e, "cg job start"));
        inner_tol_ = P_.inner_tol > 0 ? P_.inner_tol : (sizeof(WT) == 4 ? 1e-5 : P_.tol);
        // the inner iteration's vector kernels get at most one wave of
        // resident blocks each (their loops stride over the rest)
        alphaBlocks_ = resident_grid(k_cg_alpha<WT>);
        updateBlocks_ = resident_grid(k_cg_update<WT>);
        directionBlocks_ = resident_grid(k_cg_direction<WT>);
        check_ = P_.check_every > 0 ? P_.check_every : 16;
        // Graph replay needs a stream that can be captured (not the legacy
        // default stream, not synchronising with it) and no kernel tracing
        // (a replayed graph records no trace events).
        unsigned flags = 0;
        graph_ok_ = s_ != nullptr && s_ != cudaStreamLegacy && s_ != cudaStreamPerThread &&
                    cudaStreamGetFlags(s_, &flags) == cudaSuccess && (flags & cudaStreamNonBlocking) &&
                    !trace_active();
        {
            TraceScope t("k_norm2_f64", s_);
            k_norm2_f64<<<blocks_, kVecThreads, 0, s_>>>(b_, n_, partials_, S_, 1);
        }
        count_launches(1);
        return enqueue_residual();
    }

    argcsr_status advance() override {
        if (phase_ == Done || phase_ == Failed) return status_;
        const CgState &h = *hS_;
        if (phase_ == OuterCheck) {
            const double bn = sqrt(h.bnorm2);
            rel_ = bn > 0 ? sqrt(h.norm2) / bn : sqrt(h.norm2);
            if (rel_ <= P_.tol) { converged_ = true; phase_ = Done; return ARGCSR_OK; }
            if (outer_ >= P_.max_outer || inner_total_ >= P_.max_iters) { phase_ = Done; return ARGCSR_OK; }
            ++outer_;
            // reduce the inner residual by what is still missing (4x
            // margin), but not below what the working precision can reach
            const double need = rel_ > 0 ? 0.25 * P_.tol / rel_ : inner_tol_;
            const double step_tol = need > inner_tol_ ? need : inner_tol_;
            target_ = step_tol * step_tol;
            {
                TraceScope t("k_ir_start", s_);
                k_ir_start<WT><<<blocks_, kVecThreads, 0, s_>>>(r64_, r_, p_, d_, n_, partials_, S_);
            }
            count_launches(1);
            return enqueue_inner();
        }
        // InnerCheck
        if (h.rho > target_ * h.rho0 && inner_total_ < P_.max_iters) return enqueue_inner();
        {
            TraceScope t("k_ir_correct", s_);
            k_ir_correct<WT><<<blocks_, kVecThreads, 0, s_>>>(x_, d_, n_, S_);
        }
        count_launches(1);
        return enqueue_residual();
    }

    bool step_done() const override { return ev_ && cudaEventQuery(ev_) != cudaErrorNotReady; }
    argcsr_status wait_step() override {
        cudaError_t e = cudaEventSynchronize(ev_);
        return e == cudaSuccess ? ARGCSR_OK : fail(record_cuda(e, "cg job wait"));
    }
    bool finished() const override { return phase_ == Done || phase_ == Failed; }
    argcsr_status status() const override { return status_; }
    void result(argcsr_cg_result *r) const override {
        r->outer_iters = outer_;
        r->inner_iters = inner_total_;
        r->converged = converged_ ? 1 : 0;
        r->reserved = 0;
        r->rel_residual = rel_;
    }

private:
    enum Phase { OuterCheck, InnerCheck, Done, Failed };

    argcsr_status fail(argcsr_status st) {
        phase_ = Failed;
        status_ = st;
        return st;
    }

    // r = b - A x, ||r||^2, then read the state
    argcsr_status enqueue_residual() {
        argcsr_status st = op_.residual(b_, x_, r64_, s_);
        if (st != ARGCSR_OK) return fail(st);
        {
            TraceScope t("k_norm2_f64", s_);
            k_norm2_f64<<<blocks_, kVecThreads, 0, s_>>>(r64_, n_, partials_, S_, 0);
        }
        count_launches(1);
        phase_ = OuterCheck;
        return enqueue_readback();
    }

    // `check` inner CG iterations, then read the state
    argcsr_status enqueue_inner() {
        if (!inner_exec_ && trace_active()) graph_ok_ = false;   // keep traced launches visible
        argcsr_status st = graph_ok_ ? launch_inner_graph() : launch_inner();
        if (st != ARGCSR_OK) return fail(st);
        inner_total_ += check_;
        phase_ = InnerCheck;
        return enqueue_readback();
    }

    // The inner step is the same launch sequence every time: capture it
    // once into a graph and replay it (one launch instead of 4 per
    // iteration, which is what bounds small solves).
    argcsr_status launch_inner_graph() {
        if (!inner_exec_) {
            cudaError_t e = cudaStreamBeginCapture(s_, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return record_cuda(e, "cg step capture");
            argcsr_status st = launch_inner();
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(s_, &g);
            if (st == ARGCSR_OK && e != cudaSuccess) st = record_cuda(e, "cg step capture");
            if (st == ARGCSR_OK) {
                e = cudaGraphInstantiate(&inner_exec_, g, 0);
                if (e != cudaSuccess) {
                    inner_exec_ = nullptr;
                    st = record_cuda(e, "cg step instantiate");
                }
            }
            if (g) cudaGraphDestroy(g);
            // the capture counted the kernels without running them
            g_launches.fetch_sub(kernels_per_step(), std::memory_order_relaxed);
            if (st != ARGCSR_OK) return st;
        }
        cudaError_t e = cudaGraphLaunch(inner_exec_, s_);
        if (e != cudaSuccess) return record_cuda(e, "cg step launch");
        count_launches(kernels_per_step());
        return ARGCSR_OK;
    }
    uint64_t kernels_per_step() const { return 4ull * (uint64_t)check_; }

    argcsr_status launch_inner() {
        for (int k = 0; k < check_; ++k) {
            argcsr_status st = op_.apply(p_, q_, s_);
            if (st != ARGCSR_OK) return st;
            {
                TraceScope t("k_cg_alpha", s_);
                k_cg_alpha<WT><<<alphaBlocks_, kVecThreads, 0, s_>>>(p_, q_, n_, partials_, S_);
            }
            {
                TraceScope t("k_cg_update", s_);
                k_cg_update<WT><<<updateBlocks_, kVecThreads, 0, s_>>>(d_, r_, p_, q_, n_, partials_, S_);
            }
            {
                TraceScope t("k_cg_direction", s_);
                k_cg_direction<WT><<<directionBlocks_, kVecThreads, 0, s_>>>(p_, r_, n_, S_);
            }
            count_launches(3);
        }
        return ARGCSR_OK;
    }

    argcsr_status enqueue_readback() {
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(hS_, S_, sizeof(CgState), cudaMemcpyDeviceToHost, s_);
        if (e == cudaSuccess) e = cudaEventRecord(ev_, s_);
        return e == cudaSuccess ? ARGCSR_OK : fail(record_cuda(e, "cg job step"));
    }

    Operator op_;
    long long n_;
    const double *b_;
    double *x_;
    argcsr_cg_params P_;
    cudaStream_t s_;
    int blocks_;
    int alphaBlocks_ = 1, updateBlocks_ = 1, directionBlocks_ = 1;

    // blocks_, or fewer: as many blocks of `kernel` as the GPU holds at once
    template <typename K>
    int resident_grid(K kernel) const {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kVecThreads, 0) != cudaSuccess ||
            per_sm < 1)
            return blocks_;
        const long long cap = (long long)per_sm * sms;
        return (int)(blocks_ < cap ? blocks_ : cap);
    }
    WT *r_ = nullptr, *p_ = nullptr, *q_ = nullptr, *d_ = nullptr;
    double *r64_ = nullptr, *partials_ = nullptr;
    CgState *S_ = nullptr, *hS_ = nullptr;
    cudaEvent_t ev_ = nullptr;
    cudaGraphExec_t inner_exec_ = nullptr;
    bool graph_ok_ = false;
    Phase phase_ = OuterCheck;
    argcsr_status status_ = ARGCSR_OK;
    double inner_tol_ = 0, target_ = 0, rel_ = 0;
    int check_ = 16, outer_ = 0, inner_total_ = 0;
    bool converged_ = false;
};

// Run a job to the end on its stream.
argcsr_status run_to_end(CgJob &job, argcsr_cg_result *res) {
    argcsr_status st = job.start();
    while (st == ARGCSR_OK && !job.finished()) {
        st = job.wait_step();
        if (st == ARGCSR_OK) st = job.advance();
    }
    if (st == ARGCSR_OK) st = job.status();
    if (st == ARGCSR_OK && res) job.result(res);
    return st;
}

argcsr_status check_params(const argcsr_cg_params *P) {
    if (!P || !(P->tol > 0) || P->max_iters < 0 || P->max_outer < 0 || P->inner_tol < 0) return ARGCSR_EINVAL;
    return ARGCSR_OK;
}

}  // namespace

CgJob *make_cg_job(const argcsr_matrix *A, const argcsr_matrix *Ares, const double *b, double *x,
                   const argcsr_cg_params &P, cudaStream_t s) {
    Operator op;
    op.A = A;
    op.Ares = Ares ? Ares : A;
    if (A->dtype == ARGCSR_F64) return new (std::nothrow) CgJobT<double>(op, A->n_rows, b, x, P, s);
    return new (std::nothrow) CgJobT<float>(op, A->n_rows, b, x, P, s);
}

size_t cg_job_bytes(const argcsr_matrix *A) {
    return A->dtype == ARGCSR_F64 ? CgJobT<double>::bytes_for(A->n_rows) : CgJobT<float>::bytes_for(A->n_rows);
}

}  // namespace argcsr

using namespace argcsr;

extern "C" {

ARGCSR_API argcsr_status argcsr_residual(argcsr_t A, const double *d_b, const double *d_x, double *d_r,
                                         argcsr_stream_t stream) {
    if (!A || (A->n_rows > 0 && (!d_b || !d_r)) || (A->n_cols > 0 && !d_x)) return ARGCSR_EINVAL;
    if (A->n_rows == 0) return ARGCSR_OK;
    return launch_residual_f64(A, d_b, d_x, d_r, reinterpret_cast<cudaStream_t>(stream));
}

ARGCSR_API argcsr_status argcsr_cg_solve(argcsr_t A, argcsr_t A_residual, const double *d_b,
                                         double *d_x, const argcsr_cg_params *params,
                                         argcsr_stream_t stream, argcsr_cg_result *result) {
    if (!A || A->n_rows != A->n_cols) return ARGCSR_EINVAL;
    argcsr_status st = check_params(params);
    if (st != ARGCSR_OK) return st;
    const argcsr_matrix *R = A_residual ? A_residual : A;
    if (R->n_rows != A->n_rows || R->n_cols != A->n_cols) return ARGCSR_EINVAL;
    if (A->n_rows == 0) {
        if (result) *result = argcsr_cg_result{0, 0, 1, 0, 0.0};
        return ARGCSR_OK;
    }
    if (!d_b || !d_x) return ARGCSR_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    CgJob *job = make_cg_job(A, R, d_b, d_x, *params, s);
    if (!job) return ARGCSR_ENOMEM;
    st = run_to_end(*job, result);
    delete job;
    return st;
}

ARGCSR_API argcsr_status argcsr_baseline_csr_cg(int32_t n, int64_t nnz, const int32_t *d_rowPointers,
                                                const int32_t *d_columns, const double *d_values,
                                                const double *d_b, double *d_x,
                                                const argcsr_cg_params *params, argcsr_stream_t stream,
                                                argcsr_cg_result *result) {
    if (n < 0 || nnz < 0 || nnz > 0x7fffffffLL) return ARGCSR_EINVAL;
    argcsr_status st = check_params(params);
    if (st != ARGCSR_OK) return st;
    if (n == 0) {
        if (result) *result = argcsr_cg_result{0, 0, 1, 0, 0.0};
        return ARGCSR_OK;
    }
    if (!d_rowPointers || !d_b || !d_x || (nnz > 0 && (!d_columns || !d_values))) return ARGCSR_EINVAL;
    Operator op;
    op.n = n;
    op.n_cols = n;
    op.nnz = nnz;
    op.rp = d_rowPointers;
    op.cols = d_columns;
    op.vals = d_values;
    CgJobT<double> job(op, n, d_b, d_x, *params, reinterpret_cast<cudaStream_t>(stream));
    return run_to_end(job, result);
}

}  // extern "C"
