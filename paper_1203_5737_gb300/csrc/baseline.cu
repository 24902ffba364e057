// Plain CSR SpMV kernels (Section 2's format used directly), the comparison
// baseline for ARG-CSR.
//   scalar: one thread per row, a row's entries in order;
//   vector: L = 2..32 lanes per row (L from the mean row length), lanes
//           stride the row, then a shuffle reduction within the L lanes.
#include "internal.cuh"

namespace argcsr {
namespace {

template <typename VT> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };
__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(uint16_t b) { return __uint_as_float((unsigned)b << 16); }

template <typename VT>
__global__ void __launch_bounds__(256)
k_csr_scalar(int n, const int *__restrict__ rp, const int *__restrict__ cols, const VT *__restrict__ vals,
             const typename AccOf<VT>::type *__restrict__ x, typename AccOf<VT>::type *__restrict__ y) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    typename AccOf<VT>::type sum = 0;
    for (int k = rp[r]; k < rp[r + 1]; ++k) sum = fma(widen(__ldcs(vals + k)), __ldg(x + __ldcs(cols + k)), sum);
    y[r] = sum;
}

// y = A x, or y = b - A x when b is given (a solver's residual)
template <typename VT, int L>
__global__ void __launch_bounds__(256)
k_csr_vector(int n, const int *__restrict__ rp, const int *__restrict__ cols, const VT *__restrict__ vals,
             const typename AccOf<VT>::type *__restrict__ x, typename AccOf<VT>::type *__restrict__ y,
             const typename AccOf<VT>::type *__restrict__ b = nullptr) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long r = t / L;
    const int l = (int)(t % L);
    typename AccOf<VT>::type sum = 0;
    if (r < n) {
        const int a = __ldg(rp + r), b = __ldg(rp + r + 1);
        for (int k = a + l; k < b; k += L) sum = fma(widen(__ldcs(vals + k)), __ldg(x + __ldcs(cols + k)), sum);
    }
#pragma unroll
    for (int o = L / 2; o; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o, L);
    if (r < n && l == 0) y[r] = b ? b[r] - sum : sum;
}

template <typename VT>
argcsr_status launch(int n, int64_t nnz, const int *rp, const int *cols, const void *vals, int variant,
                     const void *x, void *y, cudaStream_t s, const void *b = nullptr) {
    using Acc = typename AccOf<VT>::type;
    const VT *v = static_cast<const VT *>(vals);
    const Acc *xx = static_cast<const Acc *>(x);
    Acc *yy = static_cast<Acc *>(y);
    const Acc *bb = static_cast<const Acc *>(b);
    TraceScope t(variant == 0 ? "k_csr_scalar" : "k_csr_vector", s);
    if (variant == 0) {
        k_csr_scalar<VT><<<(n + 255) / 256, 256, 0, s>>>(n, rp, cols, v, xx, yy);
    } else {
        const double mean = n ? (double)nnz / n : 0.0;
        int L = 2;
        while (L < 32 && L < mean) L <<= 1;
        const long long threads = (long long)n * L;
        const unsigned blocks = (unsigned)((threads + 255) / 256);
        switch (L) {
            case 2: k_csr_vector<VT, 2><<<blocks, 256, 0, s>>>(n, rp, cols, v, xx, yy, bb); break;
            case 4: k_csr_vector<VT, 4><<<blocks, 256, 0, s>>>(n, rp, cols, v, xx, yy, bb); break;
            case 8: k_csr_vector<VT, 8><<<blocks, 256, 0, s>>>(n, rp, cols, v, xx, yy, bb); break;
            case 16: k_csr_vector<VT, 16><<<blocks, 256, 0, s>>>(n, rp, cols, v, xx, yy, bb); break;
            default: k_csr_vector<VT, 32><<<blocks, 256, 0, s>>>(n, rp, cols, v, xx, yy, bb); break;
        }
    }
    count_launches(1);
    ARGCSR_CHECK_LAUNCH("argcsr_baseline_csr_spmv");
    return ARGCSR_OK;
}

}  // namespace

argcsr_status launch_csr_vector_f64(int32_t n, int32_t n_cols, int64_t nnz, const int32_t *rp,
                                    const int32_t *cols, const double *vals, const double *x,
                                    double *y, cudaStream_t s) {
    (void)n_cols;
    return launch<double>(n, nnz, rp, cols, vals, 1, x, y, s);
}

argcsr_status launch_csr_residual_f64(int32_t n, int32_t n_cols, int64_t nnz, const int32_t *rp,
                                      const int32_t *cols, const double *vals, const double *b,
                                      const double *x, double *r, cudaStream_t s) {
    (void)n_cols;
    return launch<double>(n, nnz, rp, cols, vals, 1, x, r, s, b);
}

}  // namespace argcsr

extern "C" ARGCSR_API argcsr_status argcsr_baseline_csr_spmv(
    int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *d_rowPointers, const int32_t *d_columns,
    const void *d_values, argcsr_dtype dtype, int32_t variant, const void *d_x, void *d_y,
    argcsr_stream_t stream) {
    if (n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL || (variant != 0 && variant != 1))
        return ARGCSR_EINVAL;
    if (n_rows == 0) return ARGCSR_OK;
    if (!d_rowPointers || !d_y || (nnz > 0 && (!d_columns || !d_values || !d_x))) return ARGCSR_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    switch (dtype) {
        case ARGCSR_F64: return argcsr::launch<double>(n_rows, nnz, d_rowPointers, d_columns, d_values, variant, d_x, d_y, s);
        case ARGCSR_F32: return argcsr::launch<float>(n_rows, nnz, d_rowPointers, d_columns, d_values, variant, d_x, d_y, s);
        case ARGCSR_BF16: return argcsr::launch<uint16_t>(n_rows, nnz, d_rowPointers, d_columns, d_values, variant, d_x, d_y, s);
    }
    return ARGCSR_EINVAL;
}
