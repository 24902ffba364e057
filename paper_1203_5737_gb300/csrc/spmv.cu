// SpMV y = A x on ARG-CSR (Section 4 of Heller & Oberhuber).
//
// Semantics follow the paper's kernel: one thread per chunk, each thread
// sums its chunk's slots in element order (element j of chunk c at
// offset + j*G + c, or the V-interleaved form), stops at the trailing
// padding (column -1), and the partial sums of a row's chunks -- the range
// [threadsMapping[r-1], threadsMapping[r]) -- are added into y[r].
//
// GB300 design:
//  * G = 32: one warp per group, eight groups per 256-thread block.  The
//    group record is one 16-byte load; the row of each chunk comes from a
//    bit mask of row ends built with one warp reduction over threadsMapping
//    (no shared memory, no block barrier); partial sums are combined with a
//    segmented shuffle reduction and the first lane of each row stores y.
//  * G = 64 / 128: one group per G threads, the paper's shared-memory
//    reduction (a row's owner thread adds its chunks' partials).
//  * values/columns are streamed with evict-first loads (each slot is read
//    once); x is gathered through the read-only path so that its lines stay
//    in L2; V > 1 turns the per-thread loads into 8/16-byte vector loads.
//  * the loop over a chunk runs in batches of four elements, the next batch
//    loaded before the current one is consumed; the first batch is issued
//    together with the threadsMapping load.  Padding is skipped per slot
//    (column -1) rather than by a whole-warp exit: with the minimal chunk
//    size some chunk of every group is full, so a warp never runs out of
//    work before the last element row.
#include <algorithm>

#include "device.cuh"
#include "internal.cuh"

namespace argcsr {
namespace {

#ifndef ARGCSR_SPMV_ELEMS
#define ARGCSR_SPMV_ELEMS 4      // elements per lane per batch
#endif
#ifndef ARGCSR_SPMV_PREFETCH
#define ARGCSR_SPMV_PREFETCH 1   // issue batch b+1 before consuming batch b
#endif
#ifndef ARGCSR_SPMV_FIXED
#define ARGCSR_SPMV_FIXED 1      // groups with C <= 8 (V = 1): exact unrolled path
#endif

// One batch: U blocks of V consecutive elements of this lane's chunk.
template <typename VT, int V, int U>
struct Batch {
    int c[U][V];
    VT v[U][V];
};

// Load blocks [b, b+U) of a chunk (block b at base + b*stride).  Blocks past
// nb, or every block when `on` is false, read as padding without a load.
// Columns and values are loaded together: a value load does not wait for
// its column.
template <typename VT, int V, int U>
__device__ __forceinline__ void load_batch(Batch<VT, V, U> &B, const int *__restrict__ cp,
                                           const VT *__restrict__ vp, long long stride, int b,
                                           int nb, bool on) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (on && b + u < nb) {
            ld_stream<int, V>(cp + (long long)(b + u) * stride, B.c[u]);
            ld_stream<VT, V>(vp + (long long)(b + u) * stride, B.v[u]);
        } else {
#pragma unroll
            for (int e = 0; e < V; ++e) { B.c[u][e] = -1; B.v[u][e] = VT(0); }
        }
    }
}

// Where x is gathered from: global memory (ldx), or a copy in shared memory
// at a 32-bit shared-window address (an explicit ld.shared).
template <typename AT>
struct XGlobal {
    const AT *__restrict__ p;
    __device__ __forceinline__ AT operator()(int c) const { return ldx(p + c); }
};
template <typename AT>
struct XShared {
    unsigned base;
    __device__ __forceinline__ AT operator()(int c) const {
        AT v;
        if constexpr (sizeof(AT) == 8)
            asm("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(base + 8u * (unsigned)c));
        else
            asm("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(base + 4u * (unsigned)c));
        return v;
    }
};

// sum += v * x[col] over a batch, in the accumulation type AT (values are
// widened exactly: bf16 -> f32 -> AT, f32 -> AT).
template <typename VT, typename AT, int V, int U, typename XG>
__device__ __forceinline__ void consume(const Batch<VT, V, U> &B, const XG &xg, AT &sum) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
        for (int e = 0; e < V; ++e)
            if (B.c[u][e] >= 0) sum = fma((AT)widen(B.v[u][e]), xg(B.c[u][e]), sum);
}

// Sum of one chunk: C/V blocks of V elements; block b of chunk c starts at
// base + b*G*V + c*V.  The first batch may already be loaded (`first`); the
// rest are loaded only by lanes that own a row.  A minimal chunk size leaves
// at least one chunk of the group full, so the loop runs all C/V blocks (the
// paper's whole-warp early exit at padding would never fire).
template <int G, typename VT, typename AT, int V, typename XG>
__device__ __forceinline__ AT
chunk_sum(const int *__restrict__ cols, const VT *__restrict__ vals, const XG &x,
          long long base, int C, bool owns, Batch<VT, V, (ARGCSR_SPMV_ELEMS + V - 1) / V> &B) {
    constexpr int U = (ARGCSR_SPMV_ELEMS + V - 1) / V;
    AT sum = 0;
    const int nb = C / V;
    const int *cp = cols + base;
    const VT *vp = vals + base;
    const long long stride = (long long)G * V;
    for (int b = 0; b < nb; b += U) {
#if ARGCSR_SPMV_PREFETCH
        Batch<VT, V, U> N;
        load_batch<VT, V, U>(N, cp, vp, stride, b + U, nb, owns);
        consume<VT, AT, V, U, XG>(B, x, sum);
        B = N;
#else
        consume<VT, AT, V, U, XG>(B, x, sum);
        load_batch<VT, V, U>(B, cp, vp, stride, b + U, nb, owns);
#endif
    }
    return sum;
}

// What is stored for a row whose product is s: s (SpMV), b - s (the
// residual of a solver) or alpha s + beta y (y not read when beta is 0).
// MODE is a compile-time constant, so the plain product's kernel carries
// none of the others' code.
template <typename AT>
struct Epi {
    const AT *b;
    AT alpha, beta;
    template <int MODE>   // 0 product, 1 residual, 2 axpby
    __device__ __forceinline__ AT apply(AT s, const AT *__restrict__ y, long long r) const {
        if constexpr (MODE == 0) return s;
        else if constexpr (MODE == 1) return b[r] - s;
        else return beta == AT(0) ? alpha * s : fma(alpha, s, beta * y[r]);
    }
};

// Row map of a G = 32 group from threadsMapping: bit k of `ends` is set when
// chunk k is the last chunk of a row.
struct RowEnds {
    unsigned ends, below;
    int row;
    bool owns;
    __device__ __forceinline__ RowEnds(const int *__restrict__ tm, int first, int size, int lane) {
        const int end = lane < size ? __ldg(tm + first + lane) : 0;
        ends = __reduce_or_sync(FULL, lane < size ? 1u << (end - 1) : 0u);
        below = ends & ((1u << lane) - 1u);
        row = __popc(below);          // local row of this lane's chunk
        owns = row < size;            // false for free chunks
    }
};

// Segmented tree reduction of the partial sums into the first lane of each
// row, then the store: a row of t chunks costs t - 1 FP64 adds (FP64
// throughput on GB300 is about 2 operations per clock per SM, the same
// budget the FMAs use), in ceil(log2(longest row's chunk count)) steps --
// none when every row of the group has a single chunk.
template <int MODE, typename AT>
__device__ __forceinline__ void reduce_store(AT sum, const RowEnds &m, int first, int lane,
                                             const Epi<AT> &ep, AT *__restrict__ y) {
    const int segStart = m.below ? 32 - __clz(m.below) : 0;
    const unsigned atOrAbove = m.ends & ~((1u << lane) - 1u);
    const int segEnd = atOrAbove ? __ffs(atOrAbove) : 0;   // one past the row's last chunk
    const int maxChunks = __reduce_max_sync(FULL, m.owns ? segEnd - segStart : 0);
    for (int o = 1; o < maxChunks; o <<= 1) {
        const AT v = __shfl_down_sync(FULL, sum, o);
        add_if(sum, v, ((lane - segStart) & (2 * o - 1)) == 0 && lane + o < segEnd);
    }
    if (m.owns && lane == segStart) y[first + m.row] = ep.template apply<MODE>(sum, y, first + m.row);
}

// A group whose chunk size is exactly CC (V = 1, CC <= 8): the lane issues
// all its slot loads at once, before threadsMapping is known, then all its
// x gathers, and spends no multiply-add on slot rows past the chunk.  The
// multiply-adds run in slot order, as in the batched loop.
template <int CC, int MODE, typename VT, typename AT, typename XG>
__device__ __forceinline__ void group_fixed(const int4 info, const int *__restrict__ tm,
                                            const int *__restrict__ cols, const VT *__restrict__ vals,
                                            const XG &x, const Epi<AT> &ep,
                                            AT *__restrict__ y, int lane) {
    const long long base = (long long)info.z + lane;
    int c[CC];
    VT v[CC];
#pragma unroll
    for (int j = 0; j < CC; ++j) {
        int cc[1];
        VT vv[1];
        ld_stream<int, 1>(cols + base + 32LL * j, cc);
        ld_stream<VT, 1>(vals + base + 32LL * j, vv);
        c[j] = cc[0];
        v[j] = vv[0];
    }
    const RowEnds m(tm, info.x, info.y, lane);
    AT xv[CC];
#pragma unroll
    for (int j = 0; j < CC; ++j) xv[j] = (m.owns && c[j] >= 0) ? x(c[j]) : AT(0);
    AT sum = 0;
#pragma unroll
    for (int j = 0; j < CC; ++j)
        if (m.owns && c[j] >= 0) sum = fma((AT)widen(v[j]), xv[j], sum);
    reduce_store<MODE, AT>(sum, m, info.x, lane, ep, y);
}

// G = 32: one warp per group.
// y = A x, or y = b - A x when b is given (the residual of a solver).
// A long group (G = 32, V = 1, chunk size above kLongChunk) on a whole
// block (the first blocks of k_spmv_g32, so that they start at once and run
// beside the other groups): warp w sums slot rows [w C / 8, (w + 1) C / 8) of every chunk (lane),
// in element order; the 8 partial sums of a chunk are then added in warp
// order, and the rows' chunks reduced as in k_spmv_g32.  The sums are split
// in 8 where the one-warp loop keeps one, so the result can differ from it
// in rounding (both stay within the summation bound the tests check).
template <typename VT, typename AT, int MODE>
__device__ __forceinline__ void long_group_block(const int4 info, const int *__restrict__ tm,
                                                 const int *__restrict__ cols, const VT *__restrict__ vals,
                                                 const AT *__restrict__ x, const Epi<AT> &ep,
                                                 AT *__restrict__ y) {
    __shared__ AT partial[8][32];
    constexpr int U = ARGCSR_SPMV_ELEMS;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int C = info.w;
    const int j0 = (int)((long long)C * warp / 8), j1 = (int)((long long)C * (warp + 1) / 8);
    const long long base = (long long)info.z + lane + 32LL * j0;
    const int *cp = cols + base;
    const VT *vp = vals + base;
    const int nb = j1 - j0;
    AT sum = 0;
    Batch<VT, 1, U> B;
    load_batch<VT, 1, U>(B, cp, vp, 32LL, 0, nb, true);
    for (int b = 0; b < nb; b += U) {
        Batch<VT, 1, U> N;
        load_batch<VT, 1, U>(N, cp, vp, 32LL, b + U, nb, true);
        consume<VT, AT, 1, U, XGlobal<AT>>(B, XGlobal<AT>{x}, sum);
        B = N;
    }
    partial[warp][lane] = sum;
    __syncthreads();
    if (warp != 0) return;
    AT s = partial[0][lane];
#pragma unroll
    for (int w = 1; w < 8; ++w) s += partial[w][lane];
    const RowEnds m(tm, info.x, info.y, lane);
    reduce_store<MODE, AT>(m.owns ? s : AT(0), m, info.x, lane, ep, y);
}

// Register budgets: 32, so that 64 warps fit on an SM (the gathers need
// every warp in flight), with FP32 accumulation, and with FP64 for V = 1
// when most groups take the unrolled path (WIDE false; a few registers
// spill to L1, and 40 registers with 48 warps were 5 % slower on both bench
// matrices).  The loop for chunks above 8 spills too much at 32, so
// matrices whose mean chunk size is above 8 get 40 (WIDE true), as do FP64
// V = 2; V = 4, whose wider loads need more, gets 51.
// One G = 32 group on one warp (info = its record).
template <typename VT, typename AT, int V, int MODE>
__device__ __forceinline__ void group_g32(const int4 info, const int *__restrict__ tm,
                                          const int *__restrict__ cols, const VT *__restrict__ vals,
                                          const AT *__restrict__ x, const Epi<AT> &ep, AT *__restrict__ y,
                                          int nLong, int lane) {
    constexpr int U = (ARGCSR_SPMV_ELEMS + V - 1) / V;
    const int first = info.x, size = info.y, C = info.w;
    const XGlobal<AT> xg{x};
#if ARGCSR_SPMV_FIXED
    if constexpr (V == 1) {
        switch (C) {   // warp-uniform
            case 1: group_fixed<1, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 2: group_fixed<2, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 3: group_fixed<3, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 4: group_fixed<4, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 5: group_fixed<5, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 6: group_fixed<6, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 7: group_fixed<7, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            case 8: group_fixed<8, MODE>(info, tm, cols, vals, xg, ep, y, lane); return;
            default: break;
        }
    }
#endif
    if (nLong > 0 && C > kLongChunk) return;   // done by one of the first blocks (warp-uniform)
    const long long base = (long long)info.z + lane * V;
    // the first batch does not depend on threadsMapping: issue it together
    Batch<VT, V, U> B;
    load_batch<VT, V, U>(B, cols + base, vals + base, 32LL * V, 0, C / V, true);
    const RowEnds m(tm, first, size, lane);
    AT sum = chunk_sum<32, VT, AT, V>(cols, vals, xg, base, C, m.owns, B);
    reduce_store<MODE, AT>(sum, m, first, lane, ep, y);
}

// G = 32: one warp per group.
// y = A x, or y = b - A x when b is given (the residual of a solver).
// Register budgets: 32, so that 64 warps fit on an SM (the gathers need
// every warp in flight), with FP32 accumulation, and with FP64 for V = 1
// when most groups take the unrolled path (WIDE false; a few registers
// spill to L1, and 40 registers with 48 warps were 5 % slower on both bench
// matrices).  The loop for chunks above 8 spills too much at 32, so
// matrices whose mean chunk size is above 8 get 40 (WIDE true), as do FP64
// V = 2; V = 4, whose wider loads need more, gets 51.
template <typename VT, typename AT, int V, int MODE, bool WIDE>
__global__ void __launch_bounds__(256, sizeof(AT) == 4 ? 8 : (V == 1 && !WIDE ? 8 : V == 4 ? 5 : 6))
k_spmv_g32(long long nGroups, const int4 *__restrict__ gi, const int *__restrict__ tm,
           const int *__restrict__ cols, const VT *__restrict__ vals, const AT *__restrict__ x,
           const Epi<AT> ep, AT *__restrict__ y, const int *__restrict__ longList, int nLong) {
    const int lane = threadIdx.x & 31;
    if constexpr (V == 1) {
        if ((int)blockIdx.x < nLong) {   // block-uniform: the long groups first
            long_group_block<VT, AT, MODE>(__ldg(gi + __ldg(longList + blockIdx.x)), tm, cols, vals, x, ep, y);
            return;
        }
    }
    const long long g = (long long)(blockIdx.x - nLong) * 8 + (threadIdx.x >> 5);
    if (g >= nGroups) return;  // warp-uniform
    group_g32<VT, AT, V, MODE>(__ldg(gi + g), tm, cols, vals, x, ep, y, nLong, lane);
}

// G = 64 or 128: one group per G threads, 256 / G groups per block.
template <int G, typename VT, typename AT, int V, int MODE>
__global__ void __launch_bounds__(256)
k_spmv_block(long long nGroups, const int4 *__restrict__ gi, const int *__restrict__ tm,
             const int *__restrict__ cols, const VT *__restrict__ vals, const AT *__restrict__ x,
             const Epi<AT> ep, AT *__restrict__ y) {
    using Acc = AT;
    constexpr int GPB = 256 / G;
    __shared__ Acc partial[256];
    __shared__ int rowOf[256];
    const int sub = threadIdx.x / G, c = threadIdx.x % G;
    const long long g = (long long)blockIdx.x * GPB + sub;
    const bool valid = g < nGroups;
    const int4 info = valid ? __ldg(gi + g) : make_int4(0, 0, 0, 0);
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
    constexpr int U = (ARGCSR_SPMV_ELEMS + V - 1) / V;
    const long long base = (long long)info.z + c * V;
    Batch<VT, V, U> B;
    load_batch<VT, V, U>(B, cols + base, vals + base, (long long)G * V, 0, C / V, owns);
    partial[threadIdx.x] = chunk_sum<G, VT, AT, V>(cols, vals, XGlobal<AT>{x}, base, C, owns, B);
    __syncthreads();
    if (c < size) {
        Acc s = partial[sub * G + begin];
        for (int k = begin + 1; k < end; ++k) s += partial[sub * G + k];
        y[first + c] = ep.template apply<MODE>(s, y, first + c);
    }
}

template <typename VT, typename AT, int V, int MODE, bool WIDE>
void launch_g32(long long ng, const int4 *gi, const int *tm, const int *cols, const VT *vals, const AT *x,
                const Epi<AT> &ep, AT *y, const int *longList, int nLong, cudaStream_t s) {
    k_spmv_g32<VT, AT, V, MODE, WIDE><<<(unsigned)((ng + 7) / 8 + nLong), 256, 0, s>>>(
        ng, gi, tm, cols, vals, x, ep, y, longList, nLong);
}

template <typename VT, typename AT, int V, int MODE>
argcsr_status launch_typed(const argcsr_matrix *A, const void *x, const Epi<AT> &ep, void *y,
                           cudaStream_t s) {
    const long long ng = A->n_groups;
    const auto *gi = A->d_groupInfo;
    const auto *tm = A->d_threadsMapping;
    const auto *cols = A->d_columns;
    const auto *vals = static_cast<const VT *>(A->d_values);
    const auto *xx = static_cast<const AT *>(x);
    auto *yy = static_cast<AT *>(y);
    static const char *names[2][3] = {{"k_spmv_g32", "k_residual_g32", "k_spmv_axpby_g32"},
                                      {"k_spmv_block", "k_residual_block", "k_spmv_axpby_block"}};
    TraceScope t(names[A->G == 32 ? 0 : 1][MODE], s);
    const int nLong = V == 1 && A->G == 32 ? (int)A->n_long : 0;
    switch (A->G) {
        case 32: {
            bool wide = false;
            // FP64, V = 1, mean chunk size S / (32 groups) above 8: mostly the looped path
            if constexpr (sizeof(AT) == 8 && V == 1) wide = A->n_slots > 8LL * 32 * ng;
            if constexpr (sizeof(AT) == 8 && V == 1) {
                if (wide) {
                    launch_g32<VT, AT, V, MODE, true>(ng, gi, tm, cols, vals, xx, ep, yy, A->d_longGroups,
                                                      nLong, s);
                    break;
                }
            }
            launch_g32<VT, AT, V, MODE, false>(ng, gi, tm, cols, vals, xx, ep, yy, A->d_longGroups, nLong, s);
            break;
        }
        case 64: k_spmv_block<64, VT, AT, V, MODE><<<(unsigned)((ng + 3) / 4), 256, 0, s>>>(ng, gi, tm, cols, vals, xx, ep, yy); break;
        default: k_spmv_block<128, VT, AT, V, MODE><<<(unsigned)((ng + 1) / 2), 256, 0, s>>>(ng, gi, tm, cols, vals, xx, ep, yy); break;
    }
    count_launches(1);
    ARGCSR_CHECK_LAUNCH("argcsr_spmv kernel");
    return ARGCSR_OK;
}

template <typename VT, typename AT, int MODE>
argcsr_status launch_v(const argcsr_matrix *A, const void *x, const Epi<AT> &ep, void *y, cudaStream_t s) {
    switch (A->V) {
        case 1: return launch_typed<VT, AT, 1, MODE>(A, x, ep, y, s);
        case 2: return launch_typed<VT, AT, 2, MODE>(A, x, ep, y, s);
        default: return launch_typed<VT, AT, 4, MODE>(A, x, ep, y, s);
    }
}

template <typename AT>
Epi<AT> epi(const void *b = nullptr, double alpha = 1.0, double beta = 0.0) {
    return Epi<AT>{static_cast<const AT *>(b), (AT)alpha, (AT)beta};
}

// One G = 32 group of a batch member on one warp (k = 1, V = 1), gathering x
// through xg: the single-matrix product's code, a long group included.
template <typename VT, typename AT, typename XG>
__device__ __forceinline__ void batch_group(const int4 info, const int *__restrict__ tm,
                                            const int *__restrict__ cols, const VT *__restrict__ vals,
                                            const XG &xg, AT *__restrict__ y, int lane) {
    const Epi<AT> ep{nullptr, AT(1), AT(0)};
    switch (info.w) {   // warp-uniform
        case 1: group_fixed<1, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 2: group_fixed<2, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 3: group_fixed<3, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 4: group_fixed<4, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 5: group_fixed<5, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 6: group_fixed<6, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 7: group_fixed<7, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        case 8: group_fixed<8, 0>(info, tm, cols, vals, xg, ep, y, lane); return;
        default: break;
    }
    constexpr int U = ARGCSR_SPMV_ELEMS;
    const long long base = (long long)info.z + lane;
    Batch<VT, 1, U> B;
    load_batch<VT, 1, U>(B, cols + base, vals + base, 32LL, 0, info.w, true);
    const RowEnds rm(tm, info.x, info.y, lane);
    const AT sum = chunk_sum<32, VT, AT, 1>(cols, vals, xg, base, info.w, rm.owns, B);
    reduce_store<0, AT>(sum, rm, info.x, lane, ep, y);
}

// Every group of a batch of matrices (k = 1, V = 1): one block of 32 warps
// per matrix, the matrices with the most slots first (`order`), the
// matrix's groups shared out among the warps.  When the matrix's x fits the
// block's shared memory (at most xCap elements) it is copied there once and
// gathered from there: a warp's 32 random shared-memory reads cost a few
// bank wavefronts, where 32 random global reads cost 32 L1 wavefronts even
// when they hit, and those wavefronts are what bounds a product whose x
// stays on chip.  Larger members gather from global memory.
template <typename VT, typename AT>
__global__ void __launch_bounds__(1024, sizeof(AT) == 4 ? 2 : 1)
k_batch_spmv_g32(const BatchDesc *__restrict__ desc, const int *__restrict__ order, int xCap,
                 const AT *__restrict__ X, AT *__restrict__ Y) {
    extern __shared__ __align__(16) unsigned char xsm[];
    const int m = __ldg(order + blockIdx.x);
    const BatchDesc d = desc[m];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const AT *x = X + d.colBase;
    AT *y = Y + d.rowBase;
    const VT *vals = static_cast<const VT *>(d.vals);
    if (d.nCols <= xCap) {   // block-uniform
        AT *xs = reinterpret_cast<AT *>(xsm);
        for (int i = threadIdx.x; i < d.nCols; i += 1024) xs[i] = __ldg(x + i);
        __syncthreads();
        const XShared<AT> xg{(unsigned)__cvta_generic_to_shared(xsm)};
        for (long long g = warp; g < d.nGroups; g += 32)
            batch_group<VT, AT>(__ldg(d.gi + g), d.tm, d.cols, vals, xg, y, lane);
    } else {
        const XGlobal<AT> xg{x};
        for (long long g = warp; g < d.nGroups; g += 32)
            batch_group<VT, AT>(__ldg(d.gi + g), d.tm, d.cols, vals, xg, y, lane);
    }
}

// Roofline probe: the memory accesses of k_spmv_g32 (G = 32, V = 1) without
// its arithmetic.  Per group one record load, then for every slot row the
// column stream (MODE 0 and 2), the value stream as well (MODE 1), and for
// every column >= 0 one gather of x with load instruction OP (MODE 0 and 1;
// MODE 2 reads the columns only).  The loaded bits are XOR-folded per lane
// in integer registers and stored only if they equal a constant that no
// input produces by chance: in practice nothing is written, and no load can
// be dropped.  No FP64 instruction is issued.
__device__ unsigned long long g_probe_sink;

template <int MODE, int OP, int V>
__global__ void __launch_bounds__(256, 8)
k_probe_g32(long long nGroups, const int4 *__restrict__ gi, const int *__restrict__ cols,
            const double *__restrict__ vals, const double *__restrict__ x, const int *__restrict__ longList,
            int nLong) {
    constexpr int U = (ARGCSR_SPMV_ELEMS + V - 1) / V;   // V-blocks per batch
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // the product's split of the work: the long groups (V = 1) first, one per
    // block with its slot rows shared out among the 8 warps, then one group
    // per warp
    int4 info;
    int j0, nb;
    if (V == 1 && (int)blockIdx.x < nLong) {   // block-uniform
        info = __ldg(gi + __ldg(longList + blockIdx.x));
        j0 = (int)((long long)info.w * warp / 8);
        nb = (int)((long long)info.w * (warp + 1) / 8);
    } else {
        const long long g = (long long)(blockIdx.x - nLong) * 8 + warp;
        if (g >= nGroups) return;   // warp-uniform
        info = __ldg(gi + g);
        if (nLong > 0 && info.w > kLongChunk) return;   // done by one of the first blocks
        j0 = 0;
        nb = info.w / V;
    }
    const long long base = (long long)info.z + lane * V;
    unsigned long long acc = 0;
    for (int j = j0; j < nb; j += U) {
        int c[U][V];
        double v[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int e = 0; e < V; ++e) { c[u][e] = -1; v[u][e] = 0.0; }
            if (j + u < nb) {
                ld_stream<int, V>(cols + base + 32LL * V * (j + u), c[u]);
                if constexpr (MODE == 1) ld_stream<double, V>(vals + base + 32LL * V * (j + u), v[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                if constexpr (MODE == 2) {
                    acc ^= (unsigned)c[u][e];
                } else if (c[u][e] >= 0) {
                    acc ^= (unsigned long long)__double_as_longlong(ldx<OP>(x + c[u][e]));
                    if constexpr (MODE == 1) acc ^= (unsigned long long)__double_as_longlong(v[u][e]);
                }
            }
    }
    if (acc == 0x5a5a5a5a5a5a5a5aULL) g_probe_sink = acc;
}

// The probe for G = 64 or 128 layouts, in k_spmv_block's split: one group
// per G threads, thread c reading chunk c (V-blocks G V apart).
template <int G, int MODE, int V>
__global__ void __launch_bounds__(256)
k_probe_block(long long nGroups, const int4 *__restrict__ gi, const int *__restrict__ cols,
              const double *__restrict__ vals, const double *__restrict__ x) {
    constexpr int U = (ARGCSR_SPMV_ELEMS + V - 1) / V;
    const int sub = threadIdx.x / G, c = threadIdx.x % G;
    const long long g = (long long)blockIdx.x * (256 / G) + sub;
    if (g >= nGroups) return;   // uniform over the group's G threads (whole warps)
    const int4 info = __ldg(gi + g);
    const long long base = (long long)info.z + c * V;
    const int nb = info.w / V;
    unsigned long long acc = 0;
    for (int j = 0; j < nb; j += U) {
        int cc[U][V];
        double v[U][V];
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int e = 0; e < V; ++e) { cc[u][e] = -1; v[u][e] = 0.0; }
            if (j + u < nb) {
                ld_stream<int, V>(cols + base + (long long)G * V * (j + u), cc[u]);
                if constexpr (MODE == 1) ld_stream<double, V>(vals + base + (long long)G * V * (j + u), v[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                if constexpr (MODE == 2) {
                    acc ^= (unsigned)cc[u][e];
                } else if (cc[u][e] >= 0) {
                    acc ^= (unsigned long long)__double_as_longlong(ldx<0>(x + cc[u][e]));
                    if constexpr (MODE == 1) acc ^= (unsigned long long)__double_as_longlong(v[u][e]);
                }
            }
    }
    if (acc == 0x5a5a5a5a5a5a5a5aULL) g_probe_sink = acc;
}

template <int G, int V>
void launch_probe_block(const argcsr_matrix *A, const double *x, int what, cudaStream_t s) {
    const unsigned blocks = (unsigned)((A->n_groups + 256 / G - 1) / (256 / G));
    const auto *v = static_cast<const double *>(A->d_values);
    if (what == 0) k_probe_block<G, 0, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x);
    else if (what == 1) k_probe_block<G, 1, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x);
    else k_probe_block<G, 2, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x);
}

template <int G>
void launch_probe_block_v(const argcsr_matrix *A, const double *x, int what, cudaStream_t s) {
    if (A->V == 1) launch_probe_block<G, 1>(A, x, what, s);
    else if (A->V == 2) launch_probe_block<G, 2>(A, x, what, s);
    else launch_probe_block<G, 4>(A, x, what, s);
}

template <int MODE, int V>
void launch_probe_mode(unsigned blocks, const argcsr_matrix *A, const double *x, int op, int nLong,
                       cudaStream_t s) {
    const auto *v = static_cast<const double *>(A->d_values);
    switch (op) {
        case 0: k_probe_g32<MODE, 0, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x,
                                                                    A->d_longGroups, nLong); break;
        case 1: k_probe_g32<MODE, 1, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x,
                                                                    A->d_longGroups, nLong); break;
        case 2: k_probe_g32<MODE, 2, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x,
                                                                    A->d_longGroups, nLong); break;
        default: k_probe_g32<MODE, 3, V><<<blocks, 256, 0, s>>>(A->n_groups, A->d_groupInfo, A->d_columns, v, x,
                                                                    A->d_longGroups, nLong); break;
    }
}

}  // namespace

argcsr_status launch_probe_gather(const argcsr_matrix *A, const void *x, int mode, cudaStream_t s) {
    if (A->n_groups == 0) return ARGCSR_OK;
    const int nLong = A->V == 1 ? (int)A->n_long : 0;
    const unsigned blocks = (unsigned)((A->n_groups + 7) / 8 + nLong);
    const int what = mode & 3, op = (mode >> 2) & 3;
    const double *xx = static_cast<const double *>(x);
    if (A->G != 32) {
        TraceScope t("k_probe_block", s);
        if (A->G == 64) launch_probe_block_v<64>(A, xx, what, s);
        else launch_probe_block_v<128>(A, xx, what, s);
        count_launches(1);
        ARGCSR_CHECK_LAUNCH("k_probe_block");
        return ARGCSR_OK;
    }
    TraceScope t("k_probe_g32", s);
    if (A->V == 4) {
        if (what == 0) launch_probe_mode<0, 4>(blocks, A, xx, op, nLong, s);
        else if (what == 1) launch_probe_mode<1, 4>(blocks, A, xx, op, nLong, s);
        else launch_probe_mode<2, 4>(blocks, A, xx, op, nLong, s);
    } else if (A->V == 2) {
        if (what == 0) launch_probe_mode<0, 2>(blocks, A, xx, op, nLong, s);
        else if (what == 1) launch_probe_mode<1, 2>(blocks, A, xx, op, nLong, s);
        else launch_probe_mode<2, 2>(blocks, A, xx, op, nLong, s);
    } else {
        if (what == 0) launch_probe_mode<0, 1>(blocks, A, xx, op, nLong, s);
        else if (what == 1) launch_probe_mode<1, 1>(blocks, A, xx, op, nLong, s);
        else launch_probe_mode<2, 1>(blocks, A, xx, op, nLong, s);
    }
    count_launches(1);
    ARGCSR_CHECK_LAUNCH("k_probe_g32");
    return ARGCSR_OK;
}

// Shared memory a k_batch_spmv_g32 block may give x: two blocks per SM.
constexpr int kBatchXBytes = 100 * 1024;

template <typename VT, typename AT>
argcsr_status launch_batch_spmv_t(const BatchDesc *desc, const int *order, int count, int maxCols,
                                  const void *X, void *Y, cudaStream_t s) {
    const int xCap = std::min(maxCols, kBatchXBytes / (int)sizeof(AT));
    const size_t smem = (size_t)std::max(xCap, 1) * sizeof(AT);
    k_batch_spmv_g32<VT, AT><<<(unsigned)count, 1024, smem, s>>>(desc, order, xCap, static_cast<const AT *>(X),
                                                                 static_cast<AT *>(Y));
    return ARGCSR_OK;
}

// The shared-memory limit of k_batch_spmv_g32, set once per device when a
// batch is created (never inside a stream capture).
argcsr_status prepare_batch_spmv() {
    cudaError_t e = cudaFuncSetAttribute(k_batch_spmv_g32<double, double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchXBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_spmv_g32<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kBatchXBytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batch_spmv_g32<uint16_t, float>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kBatchXBytes);
    return e == cudaSuccess ? ARGCSR_OK : record_cuda(e, "cudaFuncSetAttribute(k_batch_spmv_g32)");
}

argcsr_status launch_batch_spmv(const BatchDesc *desc, const int *order, int count, int maxCols,
                                long long totalGroups, argcsr_dtype dtype, const void *X, void *Y,
                                cudaStream_t s) {
    if (totalGroups == 0) return ARGCSR_OK;
    TraceScope t("k_batch_spmv_g32", s);
    argcsr_status st;
    switch (dtype) {
        case ARGCSR_F64: st = launch_batch_spmv_t<double, double>(desc, order, count, maxCols, X, Y, s); break;
        case ARGCSR_F32: st = launch_batch_spmv_t<float, float>(desc, order, count, maxCols, X, Y, s); break;
        default: st = launch_batch_spmv_t<uint16_t, float>(desc, order, count, maxCols, X, Y, s); break;
    }
    if (st != ARGCSR_OK) return st;
    count_launches(1);
    ARGCSR_CHECK_LAUNCH("k_batch_spmv_g32");
    return ARGCSR_OK;
}

argcsr_status launch_spmv(const argcsr_matrix *A, const void *x, void *y, cudaStream_t s) {
    if (A->n_groups == 0) return ARGCSR_OK;   // no rows
    switch (A->dtype) {
        case ARGCSR_F64: return launch_v<double, double, 0>(A, x, epi<double>(), y, s);
        case ARGCSR_F32: return launch_v<float, float, 0>(A, x, epi<float>(), y, s);
        default: return launch_v<uint16_t, float, 0>(A, x, epi<float>(), y, s);
    }
}

argcsr_status launch_spmv_axpby(const argcsr_matrix *A, double alpha, const void *x, double beta,
                                void *y, cudaStream_t s) {
    if (A->n_groups == 0) return ARGCSR_OK;
    switch (A->dtype) {
        case ARGCSR_F64: return launch_v<double, double, 2>(A, x, epi<double>(nullptr, alpha, beta), y, s);
        case ARGCSR_F32: return launch_v<float, float, 2>(A, x, epi<float>(nullptr, alpha, beta), y, s);
        default: return launch_v<uint16_t, float, 2>(A, x, epi<float>(nullptr, alpha, beta), y, s);
    }
}

argcsr_status launch_residual_f64(const argcsr_matrix *A, const double *b, const double *x,
                                  double *r, cudaStream_t s) {
    if (A->n_groups == 0) return ARGCSR_OK;
    switch (A->dtype) {
        case ARGCSR_F64: return launch_v<double, double, 1>(A, x, epi<double>(b), r, s);
        case ARGCSR_F32: return launch_v<float, double, 1>(A, x, epi<double>(b), r, s);
        default: return launch_v<uint16_t, double, 1>(A, x, epi<double>(b), r, s);
    }
}

}  // namespace argcsr
