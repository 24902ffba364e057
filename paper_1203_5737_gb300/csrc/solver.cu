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

#include "internal.cuh"

namespace argcsr {
namespace {

constexpr int kVecBlocks = 152 * 8;  // grid of the vector kernels (= number of partials)
constexpr int kUnroll = 4;           // independent elements per thread per step
constexpr int kVecThreads = 256;

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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum of v over the block (valid in thread 0).
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[kVecThreads / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kVecThreads / 32 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Every block contributes `partial`; returns true in thread 0 of the last
// block to finish, with the sum of all partials (in block order) in *total.
__device__ bool last_block_total(double partial, double *partials, unsigned *counter, double *total) {
    __shared__ bool s_last;
    const double bsum = block_sum(partial);
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
    t = block_sum(t);
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

template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_cg_alpha(const WT *__restrict__ p, const WT *__restrict__ q, long long n, double *partials,
           CgState *S) {
    WT acc = 0;
    FOR_EACH_ELEMENT(n, acc = fma(p[i], q[i], acc));
    double pq;
    if (last_block_total((double)acc, partials, &S->counter, &pq))
        S->alpha = pq != 0.0 ? S->rho / pq : 0.0;
}

// x += alpha p; r -= alpha q; then rho_new = r.r, beta = rho_new / rho.
template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_cg_update(WT *__restrict__ x, WT *__restrict__ r, const WT *__restrict__ p,
            const WT *__restrict__ q, long long n, double *partials, CgState *S) {
    const WT alpha = (WT)S->alpha;
    WT acc = 0;
    FOR_EACH_ELEMENT(n, {
        x[i] = fma(alpha, p[i], x[i]);
        const WT ri = fma(-alpha, q[i], r[i]);
        r[i] = ri;
        acc = fma(ri, ri, acc);
    });
    double rho_new;
    if (last_block_total((double)acc, partials, &S->counter, &rho_new)) {
        S->beta = S->rho != 0.0 ? rho_new / S->rho : 0.0;
        S->rho = rho_new;
    }
}

template <typename WT>
__global__ void __launch_bounds__(kVecThreads)
k_cg_direction(WT *__restrict__ p, const WT *__restrict__ r, long long n, const CgState *S) {
    const WT beta = (WT)S->beta;
    FOR_EACH_ELEMENT(n, p[i] = fma(beta, p[i], r[i]));
}

// ||v||^2 in FP64 into *out (norm2 or bnorm2 of the state).
__global__ void __launch_bounds__(kVecThreads)
k_norm2_f64(const double *__restrict__ v, long long n, double *partials, CgState *S, int which) {
    double acc = 0;
    FOR_EACH_ELEMENT(n, acc = fma(v[i], v[i], acc));
    double t;
    if (last_block_total(acc, partials, &S->counter, &t)) {
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
    if (last_block_total((double)acc, partials, &S->counter, &t)) {
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

template <typename WT>
struct Workspace {
    WT *r = nullptr, *p = nullptr, *q = nullptr, *d = nullptr;
    double *r64 = nullptr, *partials = nullptr;
    CgState *S = nullptr;
    CgState hS[1];           // host copy read at convergence checks
    cudaStream_t s;
    ~Workspace() {
        pool_free(r, s); pool_free(p, s); pool_free(q, s); pool_free(d, s);
        pool_free(r64, s); pool_free(partials, s); pool_free(S, s);
    }
};

#define SOLVER_CHECK(expr)                              \
    do {                                                \
        argcsr_status st_ = (expr);                     \
        if (st_ != ARGCSR_OK) return st_;               \
    } while (0)

template <typename WT>
argcsr_status cg_solve(const Operator &op, long long n, const double *b, double *x,
                       const argcsr_cg_params &P, cudaStream_t s, argcsr_cg_result *res) {
    Workspace<WT> w;
    w.s = s;
    const size_t vb = (size_t)n * sizeof(WT);
    SOLVER_CHECK(pool_alloc((void **)&w.r, vb, s));
    SOLVER_CHECK(pool_alloc((void **)&w.p, vb, s));
    SOLVER_CHECK(pool_alloc((void **)&w.q, vb, s));
    SOLVER_CHECK(pool_alloc((void **)&w.d, vb, s));
    SOLVER_CHECK(pool_alloc((void **)&w.r64, (size_t)n * 8, s));
    SOLVER_CHECK(pool_alloc((void **)&w.partials, (size_t)kVecBlocks * 8, s));
    SOLVER_CHECK(pool_alloc((void **)&w.S, sizeof(CgState), s));
    cudaError_t e = cudaMemsetAsync(w.S, 0, sizeof(CgState), s);
    if (e != cudaSuccess) return record_cuda(e, "cudaMemsetAsync");

    auto read_state = [&]() -> argcsr_status {
        cudaError_t er = cudaMemcpyAsync(w.hS, w.S, sizeof(CgState), cudaMemcpyDeviceToHost, s);
        if (er == cudaSuccess) er = cudaStreamSynchronize(s);
        return er == cudaSuccess ? ARGCSR_OK : record_cuda(er, "cg: read state");
    };
    const dim3 grid(kVecBlocks), block(kVecThreads);
    {
        TraceScope t("k_norm2_f64", s);
        k_norm2_f64<<<grid, block, 0, s>>>(b, n, w.partials, w.S, 1);
    }
    count_launches(1);
    int inner_total = 0, outer = 0;
    double rel = 0.0;
    bool converged = false;
    const double inner_tol = P.inner_tol > 0 ? P.inner_tol : (sizeof(WT) == 4 ? 1e-5 : P.tol);
    const int check = P.check_every > 0 ? P.check_every : 16;
    for (;;) {
        SOLVER_CHECK(op.residual(b, x, w.r64, s));
        {
            TraceScope t("k_norm2_f64", s);
            k_norm2_f64<<<grid, block, 0, s>>>(w.r64, n, w.partials, w.S, 0);
        }
        count_launches(1);
        ARGCSR_CHECK_LAUNCH("cg residual norm");
        SOLVER_CHECK(read_state());
        const double bn = sqrt(w.hS->bnorm2);
        rel = bn > 0 ? sqrt(w.hS->norm2) / bn : sqrt(w.hS->norm2);
        if (rel <= P.tol) { converged = true; break; }
        if (outer >= P.max_outer || inner_total >= P.max_iters) break;
        ++outer;
        // inner CG on A d = r / ||r||: reduce its residual by what is still
        // missing (with a 4x margin), but not below what the working
        // precision can reach (inner_tol)
        {
            TraceScope t("k_ir_start", s);
            k_ir_start<WT><<<grid, block, 0, s>>>(w.r64, w.r, w.p, w.d, n, w.partials, w.S);
        }
        count_launches(1);
        const double need = rel > 0 ? 0.25 * P.tol / rel : inner_tol;
        const double step_tol = need > inner_tol ? need : inner_tol;
        const double target = step_tol * step_tol;
        for (;;) {
            for (int k = 0; k < check; ++k) {
                SOLVER_CHECK(op.apply(w.p, w.q, s));
                {
                    TraceScope t("k_cg_alpha", s);
                    k_cg_alpha<WT><<<grid, block, 0, s>>>(w.p, w.q, n, w.partials, w.S);
                }
                {
                    TraceScope t("k_cg_update", s);
                    k_cg_update<WT><<<grid, block, 0, s>>>(w.d, w.r, w.p, w.q, n, w.partials, w.S);
                }
                {
                    TraceScope t("k_cg_direction", s);
                    k_cg_direction<WT><<<grid, block, 0, s>>>(w.p, w.r, n, w.S);
                }
                count_launches(3);
            }
            ARGCSR_CHECK_LAUNCH("cg inner iteration");
            inner_total += check;
            SOLVER_CHECK(read_state());
            const CgState &h = *w.hS;
            if (!(h.rho > target * h.rho0) || inner_total >= P.max_iters) break;
        }
        {
            TraceScope t("k_ir_correct", s);
            k_ir_correct<WT><<<grid, block, 0, s>>>(x, w.d, n, w.S);
        }
        count_launches(1);
    }
    if (res) {
        res->outer_iters = outer;
        res->inner_iters = inner_total;
        res->converged = converged ? 1 : 0;
        res->rel_residual = rel;
    }
    return ARGCSR_OK;
}

argcsr_status check_params(const argcsr_cg_params *P) {
    if (!P || !(P->tol > 0) || P->max_iters < 0 || P->max_outer < 0 || P->inner_tol < 0) return ARGCSR_EINVAL;
    return ARGCSR_OK;
}

}  // namespace
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
    Operator op;
    op.A = A;
    op.Ares = R;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (A->dtype == ARGCSR_F64) return cg_solve<double>(op, A->n_rows, d_b, d_x, *params, s, result);
    return cg_solve<float>(op, A->n_rows, d_b, d_x, *params, s, result);
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
    return cg_solve<double>(op, n, d_b, d_x, *params, reinterpret_cast<cudaStream_t>(stream), result);
}

}  // extern "C"
