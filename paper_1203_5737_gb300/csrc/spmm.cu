// Multi-right-hand-side products Y = A X on ARG-CSR, batches of matrices in
// one persistent launch, and an empirical autotuner for the format's
// parameters (G, desiredChunkSize).
//
// SpMM keeps the Section 4 kernel structure -- one thread per chunk, a
// chunk's slots in element order, partial sums combined per row -- and gives
// every slot k multiply-adds against row `col` of X.  X and Y are row-major
// (a column index selects k consecutive values), so one slot's k values of X
// come with one or a few vector loads.
//
// The batch kernel runs the G = 32 warp-per-group body over the groups of
// all matrices of a batch: warps share out the concatenated group list,
// so a launch has a fixed grid (a few blocks per SM) whatever the number and
// sizes of the matrices, and can be captured once in a CUDA graph.
#include <math.h>

#include <vector>

#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

struct argcsr_batch {
    int device;
    int32_t count;
    argcsr_dtype dtype;
    int32_t V;
    int64_t total_rows, total_cols, total_groups, total_nnz, total_slots;
    void *d_desc;                 // BatchDesc[count]
    long long *d_groupPrefix;     // count + 1
    int *d_order;                 // members by stored slots, most first (count)
    int maxCols;                  // largest member's column count
    std::vector<int64_t> rowOff, colOff;   // host prefix sums (count + 1)
};

struct argcsr_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace argcsr {
namespace {

// k values of row `col` of X (row-major, leading dimension ld).
template <typename AT, int K, bool VEC>
__device__ __forceinline__ void load_x_row(const AT *__restrict__ row, AT (&xv)[K]) {
    if constexpr (VEC && sizeof(AT) == 4 && K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q) {
            const float4 t = __ldg(reinterpret_cast<const float4 *>(row) + q);
            xv[4 * q] = t.x; xv[4 * q + 1] = t.y; xv[4 * q + 2] = t.z; xv[4 * q + 3] = t.w;
        }
    } else if constexpr (VEC && sizeof(AT) == 8 && K % 2 == 0) {
#pragma unroll
        for (int q = 0; q < K / 2; ++q) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(row) + q);
            xv[2 * q] = t.x; xv[2 * q + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) xv[q] = __ldg(row + q);
    }
}

template <typename AT, int K, bool VEC>
__device__ __forceinline__ void store_y_row(AT *__restrict__ row, const AT (&v)[K]) {
    if constexpr (VEC && sizeof(AT) == 4 && K % 4 == 0) {
#pragma unroll
        for (int q = 0; q < K / 4; ++q)
            reinterpret_cast<float4 *>(row)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int q = 0; q < K; ++q) row[q] = v[q];
    }
}

// One G = 32 group, one warp: Y[row, 0:K] = sum over the row's chunks.
template <typename VT, typename AT, int K, int V, bool VEC>
__device__ __forceinline__ void spmm_group_g32(const int4 info, const int *__restrict__ tm,
                                               const int *__restrict__ cols,
                                               const VT *__restrict__ vals,
                                               const AT *__restrict__ X, long long ldx,
                                               AT *__restrict__ Y, long long ldy, int lane) {
    const int first = info.x, size = info.y, C = info.w;
    const WarpRowMap rm(tm, first, size, lane);
    AT acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = 0;
    const long long base = (long long)info.z + lane * V;
    const int nb = C / V;
#pragma unroll 2
    for (int b = 0; b < nb; ++b) {
        int c[V];
        VT v[V];
        if (rm.owns) {
            ld_stream<int, V>(cols + base + (long long)b * 32 * V, c);
            ld_stream<VT, V>(vals + base + (long long)b * 32 * V, v);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) c[e] = -1;
        }
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if (c[e] >= 0) {
                AT xv[K];
                load_x_row<AT, K, VEC>(X + (long long)c[e] * ldx, xv);
                const AT a = (AT)widen(v[e]);
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] = fma(a, xv[q], acc[q]);
            }
        }
    }
    // segmented tree reduction into the first lane of each row
    const int maxChunks = __reduce_max_sync(FULL, rm.owns ? rm.segEnd - rm.segStart : 0);
    for (int o = 1; o < maxChunks; o <<= 1) {
        const bool on = ((lane - rm.segStart) & (2 * o - 1)) == 0 && lane + o < rm.segEnd;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const AT t = __shfl_down_sync(FULL, acc[q], o);
            add_if(acc[q], t, on);
        }
    }
    if (rm.owns && lane == rm.segStart) store_y_row<AT, K, VEC>(Y + (long long)(first + rm.row) * ldy, acc);
}

// A long group (V = 1, chunk size above kLongChunk) on a whole block, as the
// SpMV does it: warp w takes slot rows [w C / 8, (w + 1) C / 8) of every
// chunk, the 8 partial sums are added in warp order, then the rows are
// reduced.  Every column's arithmetic is the SpMV's, so column j of Y equals
// the SpMV of column j of X bit for bit here too.
template <typename VT, typename AT, int K, bool VEC>
__device__ __forceinline__ void spmm_long_block(const int4 info, const int *__restrict__ tm,
                                                const int *__restrict__ cols, const VT *__restrict__ vals,
                                                const AT *__restrict__ X, long long ldx,
                                                AT *__restrict__ Y, long long ldy) {
    __shared__ AT partial[8][32][K];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int C = info.w;
    const int j0 = (int)((long long)C * warp / 8), j1 = (int)((long long)C * (warp + 1) / 8);
    const long long base = (long long)info.z + lane;
    AT acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = 0;
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
        int c[1];
        VT v[1];
        ld_stream<int, 1>(cols + base + 32LL * j, c);
        ld_stream<VT, 1>(vals + base + 32LL * j, v);
        if (c[0] >= 0) {
            AT xv[K];
            load_x_row<AT, K, VEC>(X + (long long)c[0] * ldx, xv);
            const AT a = (AT)widen(v[0]);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[q] = fma(a, xv[q], acc[q]);
        }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) partial[warp][lane][q] = acc[q];
    __syncthreads();
    if (warp != 0) return;
#pragma unroll
    for (int q = 0; q < K; ++q) {
        acc[q] = partial[0][lane][q];
#pragma unroll
        for (int w = 1; w < 8; ++w) acc[q] += partial[w][lane][q];
    }
    const WarpRowMap rm(tm, info.x, info.y, lane);
    const int maxChunks = __reduce_max_sync(FULL, rm.owns ? rm.segEnd - rm.segStart : 0);
    for (int o = 1; o < maxChunks; o <<= 1) {
        const bool on = ((lane - rm.segStart) & (2 * o - 1)) == 0 && lane + o < rm.segEnd;
#pragma unroll
        for (int q = 0; q < K; ++q) {
            const AT t = __shfl_down_sync(FULL, acc[q], o);
            add_if(acc[q], t, on);
        }
    }
    if (rm.owns && lane == rm.segStart) store_y_row<AT, K, VEC>(Y + (long long)(info.x + rm.row) * ldy, acc);
}

template <typename VT, typename AT, int K, int V, bool VEC>
__global__ void __launch_bounds__(256)
k_spmm_g32(long long nGroups, const int4 *__restrict__ gi, const int *__restrict__ tm,
           const int *__restrict__ cols, const VT *__restrict__ vals, const AT *__restrict__ X,
           long long ldx, AT *__restrict__ Y, long long ldy, const int *__restrict__ longList, int nLong) {
    if constexpr (V == 1) {
        if ((int)blockIdx.x < nLong) {   // block-uniform: the long groups first
            spmm_long_block<VT, AT, K, VEC>(__ldg(gi + __ldg(longList + blockIdx.x)), tm, cols, vals, X, ldx, Y, ldy);
            return;
        }
    }
    const long long g = (long long)(blockIdx.x - nLong) * 8 + (threadIdx.x >> 5);
    if (g >= nGroups) return;
    const int4 info = __ldg(gi + g);
    if (nLong > 0 && info.w > kLongChunk) return;   // done by one of the first blocks (warp-uniform)
    spmm_group_g32<VT, AT, K, V, VEC>(info, tm, cols, vals, X, ldx, Y, ldy, threadIdx.x & 31);
}

// G = 64 / 128: one group per G threads, the row owner adds its chunks.
template <int G, typename VT, typename AT, int K, int V, bool VEC>
__global__ void __launch_bounds__(256)
k_spmm_block(long long nGroups, const int4 *__restrict__ gi, const int *__restrict__ tm,
             const int *__restrict__ cols, const VT *__restrict__ vals, const AT *__restrict__ X,
             long long ldx, AT *__restrict__ Y, long long ldy) {
    constexpr int GPB = 256 / G;
    __shared__ AT partial[256][K];
    __shared__ int rowOf[256];
    const int sub = threadIdx.x / G, c = threadIdx.x % G;
    const long long g = (long long)blockIdx.x * GPB + sub;
    const int4 info = g < nGroups ? __ldg(gi + g) : make_int4(0, 0, 0, 0);
    const int first = info.x, size = info.y, C = info.w;
    rowOf[threadIdx.x] = -1;
    __syncthreads();
    int begin = 0, end = 0;
    if (c < size) {
        end = __ldg(tm + first + c);
        begin = c ? __ldg(tm + first + c - 1) : 0;
        for (int k = begin; k < end; ++k) rowOf[sub * G + k] = c;
    }
    __syncthreads();
    const bool owns = rowOf[threadIdx.x] >= 0;
    AT acc[K];
#pragma unroll
    for (int q = 0; q < K; ++q) acc[q] = 0;
    const long long base = (long long)info.z + c * V;
    for (int b = 0; b < C / V; ++b) {
        if (!owns) break;
        int cc[V];
        VT v[V];
        ld_stream<int, V>(cols + base + (long long)b * G * V, cc);
        ld_stream<VT, V>(vals + base + (long long)b * G * V, v);
#pragma unroll
        for (int e = 0; e < V; ++e) {
            if (cc[e] >= 0) {
                AT xv[K];
                load_x_row<AT, K, VEC>(X + (long long)cc[e] * ldx, xv);
                const AT a = (AT)widen(v[e]);
#pragma unroll
                for (int q = 0; q < K; ++q) acc[q] = fma(a, xv[q], acc[q]);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < K; ++q) partial[threadIdx.x][q] = acc[q];
    __syncthreads();
    if (c < size) {
        AT s[K];
#pragma unroll
        for (int q = 0; q < K; ++q) s[q] = partial[sub * G + begin][q];
        for (int k = begin + 1; k < end; ++k)
#pragma unroll
            for (int q = 0; q < K; ++q) s[q] += partial[sub * G + k][q];
        store_y_row<AT, K, VEC>(Y + (long long)(first + c) * ldy, s);
    }
}

// Phases of one G = 32 group, so that a warp can interleave two groups:
// (1) issue the threadsMapping load and the group's first slot rows,
// (2) find the lane's row, gather x and accumulate (remaining slot rows
//     follow), (3) reduce per row and store.
template <typename VT, typename AT, int K, int V>
struct GroupWork {
    static constexpr int U = V >= 4 ? 1 : 4 / V;   // V-blocks loaded in phase 1
    int4 info;
    const int *tm;
    const int *cols;
    const VT *vals;
    const AT *X;
    AT *Y;
    int tmv;
    int c[U][V];
    VT v[U][V];
    AT acc[K];

    __device__ __forceinline__ void issue(int lane) {
        const int size = info.y, nb = info.w / V;
        tmv = lane < size ? __ldg(tm + info.x + lane) : 0;
        const long long base = (long long)info.z + lane * V;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (u < nb) {
                ld_stream<int, V>(cols + base + (long long)u * 32 * V, c[u]);
                ld_stream<VT, V>(vals + base + (long long)u * 32 * V, v[u]);
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) c[u][e] = -1;
            }
        }
    }
    __device__ __forceinline__ void slot(int col, VT val) {
        if (col >= 0) {
            AT xv[K];
            load_x_row<AT, K, (K % 4 == 0 || (sizeof(AT) == 8 && K % 2 == 0))>(X + (long long)col * K, xv);
            const AT a = (AT)widen(val);
#pragma unroll
            for (int q = 0; q < K; ++q) acc[q] = fma(a, xv[q], acc[q]);
        }
    }
    __device__ __forceinline__ void finish(int lane) {
        const int size = info.y, nb = info.w / V;
        const unsigned ends = __reduce_or_sync(FULL, lane < size ? 1u << (tmv - 1) : 0u);
        const unsigned below = ends & ((1u << lane) - 1u);
        const int row = __popc(below);
        const bool owns = row < size;
        const int segStart = below ? 32 - __clz(below) : 0;
        const unsigned atOrAbove = ends & ~((1u << lane) - 1u);
        const int segEnd = atOrAbove ? __ffs(atOrAbove) : 0;
#pragma unroll
        for (int q = 0; q < K; ++q) acc[q] = 0;
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int e = 0; e < V; ++e) slot(owns ? c[u][e] : -1, v[u][e]);
        const long long base = (long long)info.z + lane * V;
        for (int b = U; b < nb; ++b) {
            if (!owns) break;
            int cc[V];
            VT vv[V];
            ld_stream<int, V>(cols + base + (long long)b * 32 * V, cc);
            ld_stream<VT, V>(vals + base + (long long)b * 32 * V, vv);
#pragma unroll
            for (int e = 0; e < V; ++e) slot(cc[e], vv[e]);
        }
        const int maxChunks = __reduce_max_sync(FULL, owns ? segEnd - segStart : 0);
        for (int o = 1; o < maxChunks; o <<= 1) {
            const bool on = ((lane - segStart) & (2 * o - 1)) == 0 && lane + o < segEnd;
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const AT t = __shfl_down_sync(FULL, acc[q], o);
                add_if(acc[q], t, on);
            }
        }
        if (owns && lane == segStart)
            store_y_row<AT, K, (sizeof(AT) == 4 && K % 4 == 0)>(Y + (long long)(info.x + row) * K, acc);
    }
};

// All groups of a batch of G = 32 matrices in one launch.  Two ways to
// share the concatenated group list among the W warps of the grid:
//  * STRIPED (k >= 4): warp w takes groups w, w + W, w + 2W, ...; the warps
//    sweep the batch together, so only the few matrices under the current
//    window are live and their rows of X (k values each) stay in L1/L2;
//  * contiguous (k < 4): warp w takes one run of consecutive groups; its
//    matrix data streams in order, which wins when X rows are small.
// For k < 4 each warp works on two groups at a time (their loads are issued
// before either is consumed): batch groups are small, so the chain of
// dependent loads of a group, not bandwidth, bounds a warp.  Packed X and Y
// have leading dimension K.
template <typename VT, typename AT, int K, int V, bool STRIPED>
__global__ void __launch_bounds__(256)
k_batch_spmm_g32(const BatchDesc *__restrict__ desc, const long long *__restrict__ groupPrefix,
                 int nMat, long long totalGroups, const AT *__restrict__ X, AT *__restrict__ Y) {
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * 8;
    const long long w = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
    // matrix holding group g: last m with prefix[m] <= g (then walked forward)
    auto locate = [&](long long g) {
        int lo = 0, hi = nMat - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (groupPrefix[mid] <= g) lo = mid; else hi = mid - 1;
        }
        return lo;
    };
    auto bind = [&](GroupWork<VT, AT, K, V> &gw, long long g, int &m) {
        while (g >= groupPrefix[m + 1]) ++m;
        const BatchDesc &d = desc[m];
        gw.info = __ldg(d.gi + (g - groupPrefix[m]));
        gw.tm = d.tm;
        gw.cols = d.cols;
        gw.vals = static_cast<const VT *>(d.vals);
        gw.X = X + d.colBase * K;
        gw.Y = Y + d.rowBase * K;
    };
    // the first group of the pair runs over [gBegin, gEnd) by gStep; the
    // second is `gap` groups behind it
    // with k >= 4 a group's k sums already take many registers: one group
    // at a time keeps more warps resident (k = 4: 3.5 -> 2.7 ms, k = 16:
    // 7.6 -> 6.8 ms on the 4096-matrix batch)
    constexpr bool PAIR = K < 4;
    long long gBegin, gEnd, gStep, gap;
    if constexpr (STRIPED) {
        gBegin = w; gEnd = totalGroups; gStep = PAIR ? 2 * W : W; gap = W;
    } else {
        const long long per = (totalGroups + W - 1) / W;
        gBegin = w * per; gEnd = min(totalGroups, gBegin + per); gStep = PAIR ? 2 : 1; gap = 1;
    }
    if (gBegin >= gEnd) return;
    int ma = locate(gBegin);
    if constexpr (!PAIR) {
        GroupWork<VT, AT, K, V> a;
        for (long long g = gBegin; g < gEnd; g += gStep) {
            bind(a, g, ma);
            a.issue(lane);
            a.finish(lane);
        }
        return;
    }
    int mb = locate(min(gBegin + gap, totalGroups - 1));
    GroupWork<VT, AT, K, V> a, b;
    for (long long g = gBegin; g < gEnd; g += gStep) {
        bind(a, g, ma);
        if (g + gap < gEnd) {
            bind(b, g + gap, mb);
            a.issue(lane);
            b.issue(lane);
            a.finish(lane);
            b.finish(lane);
        } else {
            a.issue(lane);
            a.finish(lane);
        }
    }
}

// ---------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------

template <typename VT, typename AT, int K, int V, bool VEC>
void launch_spmm_kvv(const argcsr_matrix *A, const void *X, long long ldx, void *Y, long long ldy,
                     cudaStream_t s) {
    const long long ng = A->n_groups;
    const auto *vals = static_cast<const VT *>(A->d_values);
    const auto *xx = static_cast<const AT *>(X);
    auto *yy = static_cast<AT *>(Y);
    switch (A->G) {
        case 32: {
            const int nLong = V == 1 ? (int)A->n_long : 0;
            k_spmm_g32<VT, AT, K, V, VEC><<<(unsigned)((ng + 7) / 8 + nLong), 256, 0, s>>>(
                ng, A->d_groupInfo, A->d_threadsMapping, A->d_columns, vals, xx, ldx, yy, ldy, A->d_longGroups, nLong);
            break;
        }
        case 64: k_spmm_block<64, VT, AT, K, V, VEC><<<(unsigned)((ng + 3) / 4), 256, 0, s>>>(ng, A->d_groupInfo, A->d_threadsMapping, A->d_columns, vals, xx, ldx, yy, ldy); break;
        default: k_spmm_block<128, VT, AT, K, V, VEC><<<(unsigned)((ng + 1) / 2), 256, 0, s>>>(ng, A->d_groupInfo, A->d_threadsMapping, A->d_columns, vals, xx, ldx, yy, ldy); break;
    }
}

template <typename VT, typename AT, int K, bool VEC>
void launch_spmm_kv(const argcsr_matrix *A, const void *X, long long ldx, void *Y, long long ldy,
                    cudaStream_t s) {
    switch (A->V) {
        case 1: launch_spmm_kvv<VT, AT, K, 1, VEC>(A, X, ldx, Y, ldy, s); break;
        case 2: launch_spmm_kvv<VT, AT, K, 2, VEC>(A, X, ldx, Y, ldy, s); break;
        default: launch_spmm_kvv<VT, AT, K, 4, VEC>(A, X, ldx, Y, ldy, s); break;
    }
}

template <typename VT, typename AT, bool VEC>
argcsr_status launch_spmm_t(const argcsr_matrix *A, int k, const void *X, long long ldx, void *Y,
                            long long ldy, cudaStream_t s) {
    switch (k) {
        case 1: launch_spmm_kv<VT, AT, 1, VEC>(A, X, ldx, Y, ldy, s); break;
        case 2: launch_spmm_kv<VT, AT, 2, VEC>(A, X, ldx, Y, ldy, s); break;
        case 4: launch_spmm_kv<VT, AT, 4, VEC>(A, X, ldx, Y, ldy, s); break;
        case 8: launch_spmm_kv<VT, AT, 8, VEC>(A, X, ldx, Y, ldy, s); break;
        case 16: launch_spmm_kv<VT, AT, 16, VEC>(A, X, ldx, Y, ldy, s); break;
        default: return ARGCSR_ENOTSUP;
    }
    return ARGCSR_OK;
}

// Grid of the batch kernel: twice the number of 256-thread blocks that fit
// on all SMs at once.  Two waves of half-length runs balance better than one
// wave (blocks that finish early make room for the second wave).
template <typename Kern>
unsigned persistent_grid(Kern kernel) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, 0);
    return (unsigned)(2 * max(sms, 1) * max(per, 1));
}

template <typename VT, typename AT, int K>
void launch_batch_kv(const argcsr_batch *B, const void *X, void *Y, cudaStream_t s) {
    constexpr bool S = K >= 4;
    static const unsigned grids[3] = {persistent_grid(k_batch_spmm_g32<VT, AT, K, 1, S>),
                                      persistent_grid(k_batch_spmm_g32<VT, AT, K, 2, S>),
                                      persistent_grid(k_batch_spmm_g32<VT, AT, K, 4, S>)};
    const unsigned grid = grids[B->V == 1 ? 0 : B->V == 2 ? 1 : 2];
    const auto *d = static_cast<const BatchDesc *>(B->d_desc);
    const auto *xx = static_cast<const AT *>(X);
    auto *yy = static_cast<AT *>(Y);
    switch (B->V) {
        case 1: k_batch_spmm_g32<VT, AT, K, 1, S><<<grid, 256, 0, s>>>(d, B->d_groupPrefix, B->count, B->total_groups, xx, yy); break;
        case 2: k_batch_spmm_g32<VT, AT, K, 2, S><<<grid, 256, 0, s>>>(d, B->d_groupPrefix, B->count, B->total_groups, xx, yy); break;
        default: k_batch_spmm_g32<VT, AT, K, 4, S><<<grid, 256, 0, s>>>(d, B->d_groupPrefix, B->count, B->total_groups, xx, yy); break;
    }
}

template <typename VT, typename AT>
argcsr_status launch_batch_t(const argcsr_batch *B, int k, const void *X, void *Y, cudaStream_t s) {
    switch (k) {
        case 1: launch_batch_kv<VT, AT, 1>(B, X, Y, s); break;
        case 2: launch_batch_kv<VT, AT, 2>(B, X, Y, s); break;
        case 4: launch_batch_kv<VT, AT, 4>(B, X, Y, s); break;
        case 8: launch_batch_kv<VT, AT, 8>(B, X, Y, s); break;
        case 16: launch_batch_kv<VT, AT, 16>(B, X, Y, s); break;
        default: return ARGCSR_ENOTSUP;
    }
    return ARGCSR_OK;
}

bool valid_k(int k) { return k == 1 || k == 2 || k == 4 || k == 8 || k == 16; }

argcsr_status launch_spmm(const argcsr_matrix *A, int k, const void *X, long long ldx, void *Y,
                          long long ldy, cudaStream_t s) {
    if (A->n_groups == 0) return ARGCSR_OK;
    const size_t es = vec_size(A->dtype);
    const bool vec = (uintptr_t)X % 16 == 0 && (uintptr_t)Y % 16 == 0 && (ldx * es) % 16 == 0 &&
                     (ldy * es) % 16 == 0;
    TraceScope t(A->G == 32 ? "k_spmm_g32" : "k_spmm_block", s);
    argcsr_status st;
    switch (A->dtype) {
        case ARGCSR_F64: st = vec ? launch_spmm_t<double, double, true>(A, k, X, ldx, Y, ldy, s) : launch_spmm_t<double, double, false>(A, k, X, ldx, Y, ldy, s); break;
        case ARGCSR_F32: st = vec ? launch_spmm_t<float, float, true>(A, k, X, ldx, Y, ldy, s) : launch_spmm_t<float, float, false>(A, k, X, ldx, Y, ldy, s); break;
        default: st = vec ? launch_spmm_t<uint16_t, float, true>(A, k, X, ldx, Y, ldy, s) : launch_spmm_t<uint16_t, float, false>(A, k, X, ldx, Y, ldy, s); break;
    }
    if (st != ARGCSR_OK) return st;
    count_launches(1);
    ARGCSR_CHECK_LAUNCH("argcsr_spmm kernel");
    return ARGCSR_OK;
}

argcsr_status launch_batch(const argcsr_batch *B, int k, const void *X, void *Y, cudaStream_t s) {
    if (B->total_groups == 0) return ARGCSR_OK;
    if (k == 1 && B->V == 1)   // one warp per group, the single-matrix product's code
        return launch_batch_spmv(static_cast<const BatchDesc *>(B->d_desc), B->d_order, B->count, B->maxCols,
                                 B->total_groups, B->dtype, X, Y, s);
    TraceScope t("k_batch_spmm_g32", s);
    argcsr_status st;
    switch (B->dtype) {
        case ARGCSR_F64: st = launch_batch_t<double, double>(B, k, X, Y, s); break;
        case ARGCSR_F32: st = launch_batch_t<float, float>(B, k, X, Y, s); break;
        default: st = launch_batch_t<uint16_t, float>(B, k, X, Y, s); break;
    }
    if (st != ARGCSR_OK) return st;
    count_launches(1);
    ARGCSR_CHECK_LAUNCH("argcsr_batch_spmm kernel");
    return ARGCSR_OK;
}

}  // namespace

argcsr_status launch_spmm_public(const argcsr_matrix *A, int k, const void *X, long long ldx, void *Y,
                                 long long ldy, cudaStream_t s) {
    return launch_spmm(A, k, X, ldx, Y, ldy, s);
}

}  // namespace argcsr

using namespace argcsr;

extern "C" {

ARGCSR_API argcsr_status argcsr_spmm(argcsr_t A, int32_t k, const void *d_X, int64_t ldx, void *d_Y,
                                     int64_t ldy, argcsr_stream_t stream) {
    if (!A || !valid_k(k) || ldx < k || ldy < k) return ARGCSR_EINVAL;
    if (A->n_rows == 0) return ARGCSR_OK;
    if (!d_Y || (!d_X && A->n_cols > 0)) return ARGCSR_EINVAL;
    const size_t es = vec_size(A->dtype);
    const char *x0 = static_cast<const char *>(d_X), *x1 = x0 + (size_t)A->n_cols * ldx * es;
    const char *y0 = static_cast<const char *>(d_Y), *y1 = y0 + (size_t)A->n_rows * ldy * es;
    if (d_X && x0 < y1 && y0 < x1) return ARGCSR_EINVAL;
    return launch_spmm(A, k, d_X, ldx, d_Y, ldy, reinterpret_cast<cudaStream_t>(stream));
}

ARGCSR_API argcsr_status argcsr_batch_create(int32_t count, const argcsr_t *mats, argcsr_stream_t stream,
                                             argcsr_batch_t *out) {
    if (!out) return ARGCSR_EINVAL;
    *out = nullptr;
    if (count <= 0 || !mats) return ARGCSR_EINVAL;
    for (int i = 0; i < count; ++i) {
        if (!mats[i] || mats[i]->G != 32 || mats[i]->dtype != mats[0]->dtype || mats[i]->V != mats[0]->V)
            return mats[i] && mats[i]->G != 32 ? ARGCSR_ENOTSUP : ARGCSR_EINVAL;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    argcsr_batch *B = new argcsr_batch();
    cudaGetDevice(&B->device);
    B->count = count;
    B->dtype = mats[0]->dtype;
    B->V = mats[0]->V;
    std::vector<BatchDesc> desc(count);
    std::vector<long long> prefix(count + 1, 0);
    B->rowOff.assign(count + 1, 0);
    B->colOff.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        const argcsr_matrix *A = mats[i];
        desc[i] = BatchDesc{A->d_groupInfo, A->d_threadsMapping, A->d_columns, A->d_values,
                            B->rowOff[i], B->colOff[i], A->n_groups, A->n_cols, 0};
        B->maxCols = std::max(B->maxCols, (int)A->n_cols);
        prefix[i + 1] = prefix[i] + A->n_groups;
        B->rowOff[i + 1] = B->rowOff[i] + A->n_rows;
        B->colOff[i + 1] = B->colOff[i] + A->n_cols;
        B->total_nnz += A->nnz;
        B->total_slots += A->n_slots;
    }
    B->total_rows = B->rowOff[count];
    B->total_cols = B->colOff[count];
    B->total_groups = prefix[count];
    // the members with the most slots first: the k = 1 product gives each
    // member a block, and the long ones should not start last
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return mats[a]->n_slots > mats[b]->n_slots; });
    argcsr_status st = prepare_batch_spmv();
    if (st == ARGCSR_OK) st = pool_alloc(&B->d_desc, sizeof(BatchDesc) * count, s);
    if (st == ARGCSR_OK) st = pool_alloc((void **)&B->d_groupPrefix, sizeof(long long) * (count + 1), s);
    if (st == ARGCSR_OK) st = pool_alloc((void **)&B->d_order, sizeof(int) * count, s);
    cudaError_t e = cudaSuccess;
    if (st == ARGCSR_OK) e = cudaMemcpyAsync(B->d_desc, desc.data(), sizeof(BatchDesc) * count, cudaMemcpyHostToDevice, s);
    if (st == ARGCSR_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_groupPrefix, prefix.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, s);
    if (st == ARGCSR_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s);
    if (st == ARGCSR_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors go out of scope
    if (st == ARGCSR_OK && e != cudaSuccess) st = record_cuda(e, "argcsr_batch_create");
    if (st != ARGCSR_OK) {
        pool_free(B->d_desc, s);
        pool_free(B->d_groupPrefix, s);
        pool_free(B->d_order, s);
        delete B;
        return st;
    }
    *out = B;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_batch_info(argcsr_batch_t B, int64_t *total_rows, int64_t *total_cols,
                                           int64_t *total_groups, int64_t *total_nnz,
                                           int64_t *total_slots) {
    if (!B) return ARGCSR_EINVAL;
    if (total_rows) *total_rows = B->total_rows;
    if (total_cols) *total_cols = B->total_cols;
    if (total_groups) *total_groups = B->total_groups;
    if (total_nnz) *total_nnz = B->total_nnz;
    if (total_slots) *total_slots = B->total_slots;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_batch_offsets(argcsr_batch_t B, int64_t *h_row_offsets,
                                              int64_t *h_col_offsets) {
    if (!B) return ARGCSR_EINVAL;
    for (int i = 0; i <= B->count; ++i) {
        if (h_row_offsets) h_row_offsets[i] = B->rowOff[i];
        if (h_col_offsets) h_col_offsets[i] = B->colOff[i];
    }
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_batch_spmm(argcsr_batch_t B, int32_t k, const void *d_X, void *d_Y,
                                           argcsr_stream_t stream) {
    if (!B || !valid_k(k) || !d_X || !d_Y) return ARGCSR_EINVAL;
    if ((uintptr_t)d_X % 16 || (uintptr_t)d_Y % 16) return ARGCSR_EINVAL;   // vector access
    return launch_batch(B, k, d_X, d_Y, reinterpret_cast<cudaStream_t>(stream));
}

ARGCSR_API argcsr_status argcsr_batch_graph_create(argcsr_batch_t B, int32_t k, const void *d_X,
                                                   void *d_Y, argcsr_graph_t *out) {
    if (!out) return ARGCSR_EINVAL;
    *out = nullptr;
    if (!B || !valid_k(k) || !d_X || !d_Y || (uintptr_t)d_X % 16 || (uintptr_t)d_Y % 16)
        return ARGCSR_EINVAL;
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return record_cuda(e, "cudaStreamCreateWithFlags");
    argcsr_graph *G = new argcsr_graph();
    argcsr_status st = ARGCSR_OK;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        st = launch_batch(B, k, d_X, d_Y, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &G->graph);
        if (st == ARGCSR_OK && e2 != cudaSuccess) st = record_cuda(e2, "cudaStreamEndCapture");
    } else {
        st = record_cuda(e, "cudaStreamBeginCapture");
    }
    if (st == ARGCSR_OK) {
        e = cudaGraphInstantiate(&G->exec, G->graph, 0);
        if (e != cudaSuccess) st = record_cuda(e, "cudaGraphInstantiate");
    }
    cudaStreamDestroy(cs);
    if (st != ARGCSR_OK) {
        if (G->graph) cudaGraphDestroy(G->graph);
        delete G;
        return st;
    }
    *out = G;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_graph_launch(argcsr_graph_t G, argcsr_stream_t stream) {
    if (!G) return ARGCSR_EINVAL;
    cudaError_t e = cudaGraphLaunch(G->exec, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return record_cuda(e, "cudaGraphLaunch");
    count_launches(1);
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_graph_destroy(argcsr_graph_t G) {
    if (!G) return ARGCSR_OK;
    cudaGraphExecDestroy(G->exec);
    cudaGraphDestroy(G->graph);
    delete G;
    return ARGCSR_OK;
}

ARGCSR_API argcsr_status argcsr_batch_destroy(argcsr_batch_t B, argcsr_stream_t stream) {
    if (!B) return ARGCSR_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pool_free(B->d_desc, s);
    pool_free(B->d_groupPrefix, s);
    pool_free(B->d_order, s);
    delete B;
    return ARGCSR_OK;
}

// Empirical autotuning: convert with each candidate layout, time `reps`
// products on the caller's data, keep the fastest.  Candidates whose
// conversion gives the same layout size as one already timed (same G, V,
// groups and slots) are not timed again.
ARGCSR_API argcsr_status argcsr_autotune(int32_t n_rows, int32_t n_cols, int64_t nnz,
                                         const int32_t *d_rowPointers, const int32_t *d_columns,
                                         const void *d_values, argcsr_dtype dtype, int32_t k,
                                         int32_t group_size_mask, int32_t reps,
                                         argcsr_stream_t stream, argcsr_params *best,
                                         float *best_us) {
    if (!best || !valid_k(k) || n_rows <= 0 || (group_size_mask & 7) == 0 || reps < 1) return ARGCSR_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t es = vec_size(dtype);
    void *X = nullptr, *Y = nullptr;
    argcsr_status st = pool_alloc(&X, (size_t)n_cols * k * es, s);
    if (st == ARGCSR_OK) st = pool_alloc(&Y, (size_t)n_rows * k * es, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == ARGCSR_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = ARGCSR_ECUDA;
    if (st == ARGCSR_OK && X) cudaMemsetAsync(X, 0, (size_t)n_cols * k * es, s);
    const int Gs[3] = {32, 64, 128};
    const int Ds[] = {1, 2, 3, 4, 6, 8, 12, 16, 32};
    struct Seen { int G, V; int64_t groups, slots; };
    std::vector<Seen> seen;
    float bestT = INFINITY;
    argcsr_params bp{32, 1, 1, 0};
    const int modes = (group_size_mask & 8) ? 2 : 1;
    const int widths = (group_size_mask & 16) ? 2 : 1;   // bit 16: V = 2 as well
    for (int gi = 0; gi < 3 && st == ARGCSR_OK; ++gi) {
        if (!(group_size_mask & (1 << gi))) continue;
        for (int mode = 0; mode < modes; ++mode)
        for (int vw = 1; vw <= widths; ++vw)
        for (int D : Ds) {
            argcsr_params p{Gs[gi], D, vw, mode};
            argcsr_t A = nullptr;
            argcsr_status cs = argcsr_create_from_csr(n_rows, n_cols, nnz, d_rowPointers, d_columns,
                                                      d_values, dtype, &p, stream, &A);
            if (cs == ARGCSR_EOVERFLOW) continue;
            if (cs != ARGCSR_OK) { st = cs; break; }
            bool dup = false;
            for (const Seen &q : seen)
                dup |= q.G == p.group_size && q.V == p.vec_width && q.groups == A->n_groups && q.slots == A->n_slots;
            if (!dup) {
                seen.push_back({p.group_size, p.vec_width, A->n_groups, A->n_slots});
                st = k == 1 ? launch_spmv(A, X, Y, s) : launch_spmm(A, k, X, k, Y, k, s);  // warm-up
                cudaEventRecord(e0, s);
                for (int r = 0; r < reps && st == ARGCSR_OK; ++r)
                    st = k == 1 ? launch_spmv(A, X, Y, s) : launch_spmm(A, k, X, k, Y, k, s);
                cudaEventRecord(e1, s);
                cudaError_t ee = cudaEventSynchronize(e1);
                float ms = 0;
                if (ee == cudaSuccess) ee = cudaEventElapsedTime(&ms, e0, e1);
                if (ee != cudaSuccess && st == ARGCSR_OK) st = record_cuda(ee, "argcsr_autotune timing");
                const float us = ms * 1e3f / reps;
                if (st == ARGCSR_OK && us < bestT) { bestT = us; bp = p; }
            }
            argcsr_destroy(A, stream);
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pool_free(X, s);
    pool_free(Y, s);
    if (st != ARGCSR_OK) return st;
    *best = bp;
    if (best_us) *best_us = bestT;
    return ARGCSR_OK;
}

// Autotuning for a batch: every candidate desiredChunkSize converts all
// `count` matrices (G = 32, V = 1) and times `reps` batch launches; the
// fastest D is returned.  Matrix i is given by its own CSR device arrays.
ARGCSR_API argcsr_status argcsr_autotune_batch(int32_t count, const int32_t *h_n_rows,
                                               const int32_t *h_n_cols, const int64_t *h_nnz,
                                               const int32_t *const *h_rowPointers,
                                               const int32_t *const *h_columns,
                                               const void *const *h_values, argcsr_dtype dtype,
                                               int32_t k, int32_t reps, argcsr_stream_t stream,
                                               argcsr_params *best, float *best_us) {
    if (!best || count <= 0 || !valid_k(k) || reps < 1 || !h_n_rows || !h_n_cols || !h_nnz ||
        !h_rowPointers || !h_columns || !h_values)
        return ARGCSR_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int64_t rows = 0, cols = 0;
    for (int i = 0; i < count; ++i) { rows += h_n_rows[i]; cols += h_n_cols[i]; }
    const size_t es = vec_size(dtype);
    void *X = nullptr, *Y = nullptr;
    argcsr_status st = pool_alloc(&X, (size_t)cols * k * es, s);
    if (st == ARGCSR_OK) st = pool_alloc(&Y, (size_t)rows * k * es, s);
    if (st == ARGCSR_OK && X) cudaMemsetAsync(X, 0, (size_t)cols * k * es, s);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == ARGCSR_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = ARGCSR_ECUDA;
    const int Ds[] = {1, 2, 4, 8, 16, 32};
    float bestT = INFINITY;
    argcsr_params bp{32, 1, 1, 0};
    std::vector<argcsr_t> mats(count, nullptr);
    for (int D : Ds) {
        if (st != ARGCSR_OK) break;
        argcsr_params p{32, D, 1, 0};
        bool ok = true;
        for (int i = 0; i < count && st == ARGCSR_OK; ++i) {
            argcsr_status cs = argcsr_create_from_csr(h_n_rows[i], h_n_cols[i], h_nnz[i], h_rowPointers[i],
                                                      h_columns[i], h_values[i], dtype, &p, stream, &mats[i]);
            if (cs == ARGCSR_EOVERFLOW) { ok = false; break; }
            if (cs != ARGCSR_OK) st = cs;
        }
        argcsr_batch_t B = nullptr;
        if (st == ARGCSR_OK && ok) st = argcsr_batch_create(count, mats.data(), stream, &B);
        if (st == ARGCSR_OK && ok) {
            st = launch_batch(B, k, X, Y, s);   // warm-up
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps && st == ARGCSR_OK; ++r) st = launch_batch(B, k, X, Y, s);
            cudaEventRecord(e1, s);
            cudaError_t ee = cudaEventSynchronize(e1);
            float ms = 0;
            if (ee == cudaSuccess) ee = cudaEventElapsedTime(&ms, e0, e1);
            if (ee != cudaSuccess && st == ARGCSR_OK) st = record_cuda(ee, "argcsr_autotune_batch timing");
            const float us = ms * 1e3f / reps;
            if (st == ARGCSR_OK && us < bestT) { bestT = us; bp = p; }
        }
        argcsr_batch_destroy(B, stream);
        for (auto &A : mats) { argcsr_destroy(A, stream); A = nullptr; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    pool_free(X, s);
    pool_free(Y, s);
    if (st != ARGCSR_OK) return st;
    *best = bp;
    if (best_us) *best_us = bestT;
    return ARGCSR_OK;
}

}  // extern "C"
