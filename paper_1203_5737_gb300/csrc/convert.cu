// CSR -> ARG-CSR conversion (Section 3 of Heller & Oberhuber), every step in
// device kernels.
//
// The paper's grouping is a sequential scan: read rows in order, close the
// group after the row that takes its nonzero count above D*G, or before a row
// would become its (G+1)-th.  It is made parallel here without changing its
// result:
//   1. next[s] -- where a group that started at row s would end -- depends
//      only on s, and next[s] - s is in [1, G] (k_next_delta, binary search
//      in rowPointers);
//   2. the true group starts are the chain 0, next[0], next[next[0]], ...
//      Rows are cut into tiles of T rows; since consecutive starts are at
//      most G apart, the chain enters a tile at one of its first G rows.  Per
//      tile and per possible entry, k_tile_walk follows the chain through the
//      tile and records where it leaves and how many starts it met -- a
//      function on G values;
//   3. k_resolve composes those functions in tile order (one CTA), which
//      gives every tile its true entry row and the index of its first group;
//   4. k_groups walks each tile from its true entry, and for every group
//      computes the chunk size, the per-row thread counts and the group-local
//      inclusive prefix (threadsMapping), and the group's slot offset inside
//      the tile;
//   5. k_tile_scan turns the per-tile slot totals into tile offsets;
//   6. after one read-back of the totals, k_fill writes the group records and
//      copies the CSR entries chunk by chunk into the interleaved arrays.
//
// Chunk size (Section 3, step 2).  The greedy "give one more thread to the
// row with the greatest chunk filling until all G are placed" ends with the
// smallest C for which sum over rows of max(1, ceil(len/C)) <= G: every
// greedy step only splits a row whose filling is above that C, so it never
// overshoots, and it cannot stop above it because then the rows at the
// maximum would need fewer threads than they hold.  k_groups finds that C by
// binary search with warp reductions.  Each row then keeps max(1,
// ceil(len/C)) threads; threads left over stay free (the Fig. 3 example:
// "one thread remains free").
#include <stdio.h>

#include <mutex>

#include "internal.cuh"

namespace argcsr {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void flag(unsigned *status, unsigned bits) { atomicOr(status, bits); }

// ---------------------------------------------------------------------------
// 1. next[s] - s for every row s, and validation of rowPointers.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
k_next_delta(int n, long long nnz, int G, long long limit, const int *__restrict__ rp,
             uint8_t *__restrict__ delta, DeviceTotals *tot) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int a = rp[s], b = rp[s + 1];
    if (b < a || (s == 0 && a != 0) || (s == n - 1 && (long long)b != nnz))
        flag(&tot->status, kBadRowPointers);
    // the group that starts at s ends after the first row r with
    // rp[r+1] - rp[s] > limit, or at s + G, or at n
    const int e = min(s + G, n);
    int lo = s, hi = e;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)rp[mid + 1] - a > limit) hi = mid; else lo = mid + 1;
    }
    const int next = lo < e ? lo + 1 : e;
    delta[s] = (uint8_t)(next - s);
}

// Copy delta[base, base + lim) into shared memory with 16-byte loads.  The
// delta buffer is padded to 256 bytes, so the rounded-up tail stays inside.
__device__ __forceinline__ void load_tile_delta(uint8_t *d, const uint8_t *__restrict__ delta,
                                                long long base, int lim) {
    const uint4 *src = reinterpret_cast<const uint4 *>(delta + base);
    uint4 *dst = reinterpret_cast<uint4 *>(d);
    const int n16 = (lim + 15) >> 4;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// 2. Per tile and entry e < G: exit offset past the tile and starts met.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(G)
k_tile_walk(int n, int T, const uint8_t *__restrict__ delta, uint8_t *__restrict__ fn,
            int *__restrict__ cnt) {
    extern __shared__ __align__(16) uint8_t d[];
    const int k = blockIdx.x;
    const long long base = (long long)k * T;
    const int lim = (int)min((long long)T, (long long)n - base);
    load_tile_delta(d, delta, base, lim);
    __syncthreads();
    int pos = threadIdx.x, c = 0;
    while (pos < lim) { ++c; pos += d[pos]; }
    fn[(size_t)k * G + threadIdx.x] = lim == T ? (uint8_t)(pos - T) : (uint8_t)0;
    cnt[(size_t)k * G + threadIdx.x] = c;
}

// ---------------------------------------------------------------------------
// 3. Compose the tile functions in order (one CTA of 32 warps).
// ---------------------------------------------------------------------------
template <int G>
__device__ __forceinline__ void load_table(int k, int lane, const uint8_t *__restrict__ fn,
                                           const int *__restrict__ cnt, int (&f)[G / 32],
                                           int (&c)[G / 32]) {
#pragma unroll
    for (int q = 0; q < G / 32; ++q) {
        f[q] = fn[(size_t)k * G + lane + 32 * q];
        c[q] = cnt[(size_t)k * G + lane + 32 * q];
    }
}

// Look up entry p of a table spread over the warp (entry p lives in lane
// p % 32, register p / 32).
template <int G>
__device__ __forceinline__ void lookup(const int (&f)[G / 32], const int (&c)[G / 32], int p,
                                       int &fp, int &cp) {
    fp = 0; cp = 0;
#pragma unroll
    for (int q = 0; q < G / 32; ++q) {
        const int vf = __shfl_sync(FULL, f[q], p & 31);
        const int vc = __shfl_sync(FULL, c[q], p & 31);
        if ((p >> 5) == q) { fp = vf; cp = vc; }
    }
}

template <int G>
__global__ void __launch_bounds__(1024)
k_resolve(int numTiles, const uint8_t *__restrict__ fn, const int *__restrict__ cnt,
          int *__restrict__ tileEntry, int *__restrict__ tileGroupBase, DeviceTotals *tot) {
    constexpr int E = G / 32;
    __shared__ int segF[32][G];
    __shared__ int segC[32][G];
    __shared__ int segEntry[32], segBase[32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int per = (numTiles + 31) / 32;
    const int k0 = min(numTiles, w * per), k1 = min(numTiles, k0 + per);

    int pos[E], acc[E];
#pragma unroll
    for (int q = 0; q < E; ++q) { pos[q] = lane + 32 * q; acc[q] = 0; }
    for (int k = k0; k < k1; ++k) {
        int f[E], c[E];
        load_table<G>(k, lane, fn, cnt, f, c);
#pragma unroll
        for (int q = 0; q < E; ++q) {
            int fp, cp;
            lookup<G>(f, c, pos[q], fp, cp);
            acc[q] += cp;
            pos[q] = fp;
        }
    }
#pragma unroll
    for (int q = 0; q < E; ++q) { segF[w][lane + 32 * q] = pos[q]; segC[w][lane + 32 * q] = acc[q]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int entry = 0;
        long long base = 0;
        for (int v = 0; v < 32; ++v) {
            segEntry[v] = entry;
            segBase[v] = (int)base;
            base += segC[v][entry];
            entry = segF[v][entry];
        }
        tot->n_groups = base;
    }
    __syncthreads();
    int entry = segEntry[w], base = segBase[w];
    for (int k = k0; k < k1; ++k) {
        int f[E], c[E];
        load_table<G>(k, lane, fn, cnt, f, c);
        if (lane == 0) { tileEntry[k] = entry; tileGroupBase[k] = base; }
        int fp, cp;
        lookup<G>(f, c, entry, fp, cp);
        base += cp;
        entry = fp;
    }
}

// ---------------------------------------------------------------------------
// 4. Groups of a tile: chunk size, threadsMapping, slot offset in the tile.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

template <int G>
__global__ void __launch_bounds__(256)
k_groups(int n, int T, int V, const int *__restrict__ rp, const uint8_t *__restrict__ delta,
         const int *__restrict__ tileEntry, const int *__restrict__ tileGroupBase,
         int4 *__restrict__ gscratch, int *__restrict__ threadsMapping,
         long long *__restrict__ tileSlots, DeviceTotals *tot) {
    constexpr int E = G / 32;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *d = smem;                                             // T bytes
    uint16_t *starts = reinterpret_cast<uint16_t *>(smem + T);     // T entries
    long long *slots = reinterpret_cast<long long *>(smem + 3 * (size_t)T);  // T entries
    __shared__ int s_count;
    __shared__ long long s_warp[8];

    const int k = blockIdx.x;
    const long long tbase = (long long)k * T;
    const int lim = (int)min((long long)T, (long long)n - tbase);
    load_tile_delta(d, delta, tbase, lim);
    __syncthreads();
    if (threadIdx.x == 0) {
        int pos = tileEntry[k], c = 0;
        while (pos < lim) { starts[c++] = (uint16_t)pos; pos += d[pos]; }
        s_count = c;
    }
    __syncthreads();
    const int count = s_count;
    const int gbase = tileGroupBase[k];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int i = warp; i < count; i += 8) {
        const int first = (int)(tbase + starts[i]);
        const int size = d[starts[i]];
        long long len[E];
        long long nnz = 0, maxlen = 0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            const int r = lane * E + q;
            len[q] = 0;
            if (r < size) {
                const long long l = (long long)rp[first + r + 1] - rp[first + r];
                len[q] = l > 0 ? l : 0;  // a decreasing rowPointers is flagged in k_next_delta
            }
            nnz += len[q];
            maxlen = max(maxlen, len[q]);
        }
        nnz = warp_sum_ll(nnz);
#pragma unroll
        for (int o = 16; o; o >>= 1) maxlen = max(maxlen, __shfl_xor_sync(FULL, maxlen, o));
        long long C = 0;
        if (maxlen > 0) {
            long long lo = max(1LL, (nnz + G - 1) / G), hi = maxlen;
            while (lo < hi) {
                const long long mid = lo + ((hi - lo) >> 1);
                long long need = 0;
#pragma unroll
                for (int q = 0; q < E; ++q)
                    if (lane * E + q < size) need += max(1LL, (len[q] + mid - 1) / mid);
                need = warp_sum_ll(need);
                if (need <= G) hi = mid; else lo = mid + 1;
            }
            C = (lo + V - 1) / V * V;
        }
        // thread counts and the group-local inclusive prefix
        int t[E], local = 0;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            t[q] = 0;
            if (lane * E + q < size) t[q] = C == 0 ? 1 : (int)max(1LL, (len[q] + C - 1) / C);
            local += t[q];
        }
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        int prefix = incl - local;
#pragma unroll
        for (int q = 0; q < E; ++q) {
            if (lane * E + q < size) {
                prefix += t[q];
                threadsMapping[first + lane * E + q] = prefix;
            }
        }
        if (lane == 0) {
            gscratch[gbase + i] = make_int4(first, size, 0, C <= 0x7fffffffLL ? (int)C : -1);
            slots[i] = C * G;
            if (C > 0x7fffffffLL) flag(&tot->status, kSlotOverflow);
        }
    }
    __syncthreads();
    // exclusive scan of slots[0, count) -> slot offset of each group in the tile
    const int per = (count + 255) / 256;
    const int i0 = min(count, (int)threadIdx.x * per), i1 = min(count, i0 + per);
    long long mine = 0;
    for (int i = i0; i < i1; ++i) mine += slots[i];
    long long incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    long long before = 0;
    for (int v = 0; v < warp; ++v) before += s_warp[v];
    long long run = before + incl - mine;
    for (int i = i0; i < i1; ++i) {
        if (run > 0x7fffffffLL) flag(&tot->status, kSlotOverflow);
        gscratch[gbase + i].z = (int)min(run, 0x7fffffffLL);
        run += slots[i];
    }
    if (threadIdx.x == 255) {
        long long total = 0;
        for (int v = 0; v < 8; ++v) total += s_warp[v];
        tileSlots[k] = total;
    }
}

// ---------------------------------------------------------------------------
// 5. Tile slot totals -> tile offsets; total slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_tile_scan(int numTiles, const long long *__restrict__ tileSlots, long long *__restrict__ tileSlotBase,
            DeviceTotals *tot) {
    __shared__ long long s_warp[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int per = (numTiles + 1023) / 1024;
    const int i0 = min(numTiles, (int)threadIdx.x * per), i1 = min(numTiles, i0 + per);
    long long mine = 0;
    for (int i = i0; i < i1; ++i) mine += tileSlots[i];
    long long incl = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    long long before = 0;
    for (int v = 0; v < warp; ++v) before += s_warp[v];
    long long run = before + incl - mine;
    for (int i = i0; i < i1; ++i) { tileSlotBase[i] = run; run += tileSlots[i]; }
    if (threadIdx.x == 1023) {
        long long total = 0;
        for (int v = 0; v < 32; ++v) total += s_warp[v];
        tot->n_slots = total;
        if (total > 0x7fffffffLL) flag(&tot->status, kSlotOverflow);
    }
}

// ---------------------------------------------------------------------------
// 6. Group records and the chunk-wise copy (one warp per group).
// ---------------------------------------------------------------------------
template <int G, typename VT>
__global__ void __launch_bounds__(256)
k_fill(long long nGroups, int numTiles, int V, int n_cols, const int *__restrict__ tileGroupBase,
       const long long *__restrict__ tileSlotBase, const int4 *__restrict__ gscratch,
       const int *__restrict__ rp, const int *__restrict__ colsIn, const VT *__restrict__ valsIn,
       const int *__restrict__ threadsMapping, int4 *__restrict__ groupInfo,
       int *__restrict__ colsOut, VT *__restrict__ valsOut, DeviceTotals *tot) {
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    bool bad = false;
    for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); g < nGroups;
         g += warps) {
        const int4 s = gscratch[g];
        // tile of g: the last tile whose first group index is <= g
        int lo = 0, hi = numTiles - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tileGroupBase[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const long long off = tileSlotBase[lo] + s.z;
        const int first = s.x, size = s.y, C = s.w;
        if (lane == 0) groupInfo[g] = make_int4(first, size, (int)off, C);
        if (C <= 0) continue;
#pragma unroll
        for (int q = 0; q < G / 32; ++q) {
            const int c = q * 32 + lane;
            // row of chunk c: the first row whose inclusive prefix exceeds c
            int a = 0, b = size;
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (threadsMapping[first + mid] > c) b = mid; else a = mid + 1;
            }
            long long src = 0, fill = 0;
            if (a < size) {
                const int r = first + a;
                const int begin = a == 0 ? 0 : threadsMapping[r - 1];
                const long long kk = c - begin;
                const long long len = (long long)rp[r + 1] - rp[r];
                src = rp[r] + kk * C;
                fill = min((long long)C, max(0LL, len - kk * C));
            }
            for (int j = 0; j < C; ++j) {
                const long long slot = off + (long long)(j / V) * G * V + (long long)c * V + (j % V);
                int col = -1;
                VT val;
                memset(&val, 0, sizeof val);
                if (j < fill) {
                    col = colsIn[src + j];
                    val = valsIn[src + j];
                    bad |= (col < 0) | (col >= n_cols);
                }
                colsOut[slot] = col;
                valsOut[slot] = val;
            }
        }
    }
    if (__any_sync(FULL, bad) && lane == 0) flag(&tot->status, kBadColumn);
}

// Kernels for one group size.
template <int G>
struct Kernels {
    static argcsr_status run_structure(int n, int T, int numTiles, int V, const int *rp,
                                       const uint8_t *delta, uint8_t *fn, int *cnt, int *tileEntry,
                                       int *tileGroupBase, int4 *gscratch, int *tm,
                                       long long *tileSlots, long long *tileSlotBase,
                                       DeviceTotals *tot, cudaStream_t s) {
        {
            TraceScope t("k_tile_walk", s);
            k_tile_walk<G><<<numTiles, G, T, s>>>(n, T, delta, fn, cnt);
        }
        {
            TraceScope t("k_resolve", s);
            k_resolve<G><<<1, 1024, 0, s>>>(numTiles, fn, cnt, tileEntry, tileGroupBase, tot);
        }
        {
            TraceScope t("k_groups", s);
            const size_t smem = (size_t)T * 11;  // delta, starts (u16), slots (i64)
            k_groups<G><<<numTiles, 256, smem, s>>>(n, T, V, rp, delta, tileEntry, tileGroupBase,
                                                     gscratch, tm, tileSlots, tot);
        }
        {
            TraceScope t("k_tile_scan", s);
            k_tile_scan<<<1, 1024, 0, s>>>(numTiles, tileSlots, tileSlotBase, tot);
        }
        count_launches(4);
        ARGCSR_CHECK_LAUNCH("conversion structure kernels");
        return ARGCSR_OK;
    }
    template <typename VT>
    static argcsr_status run_fill(long long nGroups, int numTiles, int V, int n_cols,
                                  const int *tileGroupBase, const long long *tileSlotBase,
                                  const int4 *gscratch, const int *rp, const int *cols,
                                  const void *vals, const int *tm, int4 *gi, int *colsOut,
                                  void *valsOut, DeviceTotals *tot, cudaStream_t s) {
        if (nGroups == 0) return ARGCSR_OK;
        const long long blocks = min((nGroups + 7) / 8, 152LL * 64);
        TraceScope t("k_fill", s);
        k_fill<G, VT><<<(unsigned)blocks, 256, 0, s>>>(
            nGroups, numTiles, V, n_cols, tileGroupBase, tileSlotBase, gscratch, rp, cols,
            static_cast<const VT *>(vals), tm, gi, colsOut, static_cast<VT *>(valsOut), tot);
        count_launches(1);
        ARGCSR_CHECK_LAUNCH("k_fill");
        return ARGCSR_OK;
    }
};

template <int G>
argcsr_status set_smem_limits(int T) {
    const size_t smem = (size_t)T * 11;
    cudaError_t e = cudaFuncSetAttribute(k_groups<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return record_cuda(e, "cudaFuncSetAttribute(k_groups)");
    return ARGCSR_OK;
}

struct Scratch {
    void *p[9] = {};
    cudaStream_t s;
    ~Scratch() { for (void *q : p) pool_free(q, s); }
};

}  // namespace
}  // namespace argcsr

using namespace argcsr;

extern "C" ARGCSR_API argcsr_status argcsr_create_from_csr(
    int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *d_rowPointers,
    const int32_t *d_columns, const void *d_values, argcsr_dtype dtype, const argcsr_params *params,
    argcsr_stream_t stream, argcsr_t *out) {
    if (!out) return ARGCSR_EINVAL;
    *out = nullptr;
    if (!params || n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL) return ARGCSR_EINVAL;
    const int G = params->group_size, D = params->desired_chunk_size, V = params->vec_width;
    if ((G != 32 && G != 64 && G != 128) || D < 1 || (V != 1 && V != 2 && V != 4)) return ARGCSR_EINVAL;
    if (dtype != ARGCSR_F64 && dtype != ARGCSR_F32 && dtype != ARGCSR_BF16) return ARGCSR_EINVAL;
    if (!d_rowPointers || (nnz > 0 && (!d_columns || !d_values))) return ARGCSR_EINVAL;
    if (n_rows == 0 && nnz != 0) return ARGCSR_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    argcsr_matrix *A = new argcsr_matrix();
    cudaGetDevice(&A->device);
    A->n_rows = n_rows; A->n_cols = n_cols; A->nnz = nnz;
    A->G = G; A->D = D; A->V = V; A->dtype = dtype;
    auto fail = [&](argcsr_status st) { argcsr_destroy(A, stream); return st; };
    if (n_rows == 0) { *out = A; return ARGCSR_OK; }

    const int n = n_rows;
    const int T = n <= (1 << 25) ? 4096 : 16384;
    const int numTiles = (int)(((long long)n + T - 1) / T);
    const size_t es = dtype_size(dtype);

    Scratch sc;
    sc.s = s;
    argcsr_status st;
#define ALLOC(i, bytes) \
    if ((st = pool_alloc(&sc.p[i], (bytes), s)) != ARGCSR_OK) return fail(st)
    ALLOC(0, (size_t)n);                                   // delta
    ALLOC(1, (size_t)numTiles * G);                        // fn
    ALLOC(2, (size_t)numTiles * G * 4);                    // cnt
    ALLOC(3, (size_t)numTiles * 4);                        // tileEntry
    ALLOC(4, (size_t)numTiles * 4);                        // tileGroupBase
    ALLOC(5, (size_t)n * 16);                              // gscratch (upper bound)
    ALLOC(6, (size_t)numTiles * 8);                        // tileSlots
    ALLOC(7, (size_t)numTiles * 8);                        // tileSlotBase
    ALLOC(8, sizeof(DeviceTotals));
    if ((st = pool_alloc((void **)&A->d_threadsMapping, (size_t)n * 4, s)) != ARGCSR_OK) return fail(st);
#undef ALLOC
    uint8_t *delta = (uint8_t *)sc.p[0];
    uint8_t *fn = (uint8_t *)sc.p[1];
    int *cnt = (int *)sc.p[2], *tileEntry = (int *)sc.p[3], *tileGroupBase = (int *)sc.p[4];
    int4 *gscratch = (int4 *)sc.p[5];
    long long *tileSlots = (long long *)sc.p[6], *tileSlotBase = (long long *)sc.p[7];
    DeviceTotals *tot = (DeviceTotals *)sc.p[8];

    cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(DeviceTotals), s);
    if (e != cudaSuccess) return fail(record_cuda(e, "cudaMemsetAsync"));
    {
        TraceScope t("k_next_delta", s);
        k_next_delta<<<(n + 255) / 256, 256, 0, s>>>(n, nnz, G, (long long)D * G, d_rowPointers, delta, tot);
    }
    count_launches(1);
    {
        cudaError_t le = cudaGetLastError();
        if (le != cudaSuccess) return fail(record_cuda(le, "k_next_delta"));
    }
    switch (G) {
        case 32: st = set_smem_limits<32>(T); if (!st) st = Kernels<32>::run_structure(n, T, numTiles, V, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, A->d_threadsMapping, tileSlots, tileSlotBase, tot, s); break;
        case 64: st = set_smem_limits<64>(T); if (!st) st = Kernels<64>::run_structure(n, T, numTiles, V, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, A->d_threadsMapping, tileSlots, tileSlotBase, tot, s); break;
        default: st = set_smem_limits<128>(T); if (!st) st = Kernels<128>::run_structure(n, T, numTiles, V, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, A->d_threadsMapping, tileSlots, tileSlotBase, tot, s); break;
    }
    if (st != ARGCSR_OK) return fail(st);

    DeviceTotals h;
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(record_cuda(e, "conversion: read totals"));
    if (h.status & kBadRowPointers) return fail(ARGCSR_EINVAL);
    if (h.status & kSlotOverflow) return fail(ARGCSR_EOVERFLOW);
    A->n_groups = h.n_groups;
    A->n_slots = h.n_slots;

    if ((st = pool_alloc((void **)&A->d_groupInfo, (size_t)A->n_groups * 16, s)) != ARGCSR_OK) return fail(st);
    if ((st = pool_alloc((void **)&A->d_columns, (size_t)A->n_slots * 4, s)) != ARGCSR_OK) return fail(st);
    if ((st = pool_alloc(&A->d_values, (size_t)A->n_slots * es, s)) != ARGCSR_OK) return fail(st);

#define FILL(GG, VT)                                                                             \
    Kernels<GG>::template run_fill<VT>(A->n_groups, numTiles, V, n_cols, tileGroupBase, tileSlotBase, \
                                       gscratch, d_rowPointers, d_columns, d_values,              \
                                       A->d_threadsMapping, A->d_groupInfo, A->d_columns,         \
                                       A->d_values, tot, s)
    if (es == 8) st = G == 32 ? FILL(32, double) : G == 64 ? FILL(64, double) : FILL(128, double);
    else if (es == 4) st = G == 32 ? FILL(32, float) : G == 64 ? FILL(64, float) : FILL(128, float);
    else st = G == 32 ? FILL(32, uint16_t) : G == 64 ? FILL(64, uint16_t) : FILL(128, uint16_t);
#undef FILL
    if (st != ARGCSR_OK) return fail(st);
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(record_cuda(e, "conversion: read status"));
    if (h.status & kBadColumn) return fail(ARGCSR_EINVAL);

    A->device_bytes = (int64_t)A->n_groups * 16 + (int64_t)n * 4 + A->n_slots * (4 + (int64_t)es);
    *out = A;
    return ARGCSR_OK;
}

// ---------------------------------------------------------------------------
// argcsr_convert_noalloc: the conversion with every intermediate array in one
// file-scope device array, for callers that must not allocate device memory.
// ---------------------------------------------------------------------------
namespace argcsr {
namespace {

constexpr int kNoallocTile = 4096;                               // T for n <= 2^25
constexpr int kNoallocMaxTiles = ARGCSR_NOALLOC_MAX_ROWS / kNoallocTile;
constexpr size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
// carve-up of the scratch array (each part 256-byte aligned)
constexpr size_t kOffDelta = 0;
constexpr size_t kOffFn = kOffDelta + align256(ARGCSR_NOALLOC_MAX_ROWS);
constexpr size_t kOffCnt = kOffFn + align256((size_t)kNoallocMaxTiles * 128);
constexpr size_t kOffEntry = kOffCnt + align256((size_t)kNoallocMaxTiles * 128 * 4);
constexpr size_t kOffGroupBase = kOffEntry + align256((size_t)kNoallocMaxTiles * 4);
constexpr size_t kOffGroups = kOffGroupBase + align256((size_t)kNoallocMaxTiles * 4);
constexpr size_t kOffTileSlots = kOffGroups + align256((size_t)ARGCSR_NOALLOC_MAX_ROWS * 16);
constexpr size_t kOffTileSlotBase = kOffTileSlots + align256((size_t)kNoallocMaxTiles * 8);
constexpr size_t kOffTotals = kOffTileSlotBase + align256((size_t)kNoallocMaxTiles * 8);
constexpr size_t kNoallocBytes = kOffTotals + align256(sizeof(DeviceTotals));
static_assert(ARGCSR_NOALLOC_MAX_ROWS % kNoallocTile == 0, "whole tiles");
static_assert(kNoallocBytes == ARGCSR_NOALLOC_SCRATCH_BYTES, "header states the scratch size");

// Every GPU that loads this library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];

// Device address of the scratch array on the current device, looked up once
// per device.  The host-side name g_noalloc_scratch is not a device address.
argcsr_status noalloc_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return record_cuda(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return ARGCSR_ENOTSUP;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return record_cuda(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_noalloc_ptr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
    return ARGCSR_OK;
}

}  // namespace
}  // namespace argcsr

extern "C" ARGCSR_API argcsr_status argcsr_convert_noalloc(
    int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *d_rowPointers,
    const int32_t *d_columns, const void *d_values, argcsr_dtype dtype, const argcsr_params *params,
    int32_t *d_groupInfo, int64_t group_capacity, int32_t *d_threadsMapping,
    int32_t *d_out_columns, void *d_out_values, int64_t slot_capacity, int64_t *h_n_groups,
    int64_t *h_n_slots, argcsr_stream_t stream) {
    if (!h_n_groups || !h_n_slots) return ARGCSR_EINVAL;
    *h_n_groups = 0;
    *h_n_slots = 0;
    if (!params || n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL) return ARGCSR_EINVAL;
    if (n_rows > ARGCSR_NOALLOC_MAX_ROWS) {
        set_error_message("argcsr_convert_noalloc: n_rows exceeds ARGCSR_NOALLOC_MAX_ROWS");
        return ARGCSR_EINVAL;
    }
    const int G = params->group_size, D = params->desired_chunk_size, V = params->vec_width;
    if ((G != 32 && G != 64 && G != 128) || D < 1 || (V != 1 && V != 2 && V != 4)) return ARGCSR_EINVAL;
    if (dtype != ARGCSR_F64 && dtype != ARGCSR_F32 && dtype != ARGCSR_BF16) return ARGCSR_EINVAL;
    if (!d_rowPointers || (nnz > 0 && (!d_columns || !d_values))) return ARGCSR_EINVAL;
    if (n_rows == 0) return nnz == 0 ? ARGCSR_OK : ARGCSR_EINVAL;
    if (!d_threadsMapping || group_capacity < 0 || slot_capacity < 0) return ARGCSR_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_groupInfo) % 16) return ARGCSR_EINVAL;  // int4 records
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    unsigned char *base = nullptr;
    argcsr_status st = noalloc_scratch(&base);
    if (st != ARGCSR_OK) return st;
    uint8_t *delta = base + kOffDelta;
    uint8_t *fn = base + kOffFn;
    int *cnt = reinterpret_cast<int *>(base + kOffCnt);
    int *tileEntry = reinterpret_cast<int *>(base + kOffEntry);
    int *tileGroupBase = reinterpret_cast<int *>(base + kOffGroupBase);
    int4 *gscratch = reinterpret_cast<int4 *>(base + kOffGroups);
    long long *tileSlots = reinterpret_cast<long long *>(base + kOffTileSlots);
    long long *tileSlotBase = reinterpret_cast<long long *>(base + kOffTileSlotBase);
    DeviceTotals *tot = reinterpret_cast<DeviceTotals *>(base + kOffTotals);

    const int n = n_rows, T = kNoallocTile;
    const int numTiles = (n + T - 1) / T;
    // the totals accumulate with atomics: they must start at zero every call
    cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(DeviceTotals), s);
    if (e != cudaSuccess) return record_cuda(e, "cudaMemsetAsync");
    {
        TraceScope t("k_next_delta", s);
        k_next_delta<<<(n + 255) / 256, 256, 0, s>>>(n, nnz, G, (long long)D * G, d_rowPointers, delta, tot);
    }
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return record_cuda(e, "k_next_delta");
    switch (G) {
        case 32: st = set_smem_limits<32>(T); if (!st) st = Kernels<32>::run_structure(n, T, numTiles, V, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, d_threadsMapping, tileSlots, tileSlotBase, tot, s); break;
        case 64: st = set_smem_limits<64>(T); if (!st) st = Kernels<64>::run_structure(n, T, numTiles, V, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, d_threadsMapping, tileSlots, tileSlotBase, tot, s); break;
        default: st = set_smem_limits<128>(T); if (!st) st = Kernels<128>::run_structure(n, T, numTiles, V, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, d_threadsMapping, tileSlots, tileSlotBase, tot, s); break;
    }
    if (st != ARGCSR_OK) return st;
    DeviceTotals h;
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda(e, "argcsr_convert_noalloc: read totals");
    if (h.status & kBadRowPointers) return ARGCSR_EINVAL;
    if (h.status & kSlotOverflow) return ARGCSR_EOVERFLOW;
    *h_n_groups = h.n_groups;
    *h_n_slots = h.n_slots;
    if (h.n_groups > group_capacity || h.n_slots > slot_capacity) {
        set_error_message("argcsr_convert_noalloc: output capacity too small (required sizes returned)");
        return ARGCSR_EINVAL;
    }
    if ((h.n_groups > 0 && !d_groupInfo) || (h.n_slots > 0 && (!d_out_columns || !d_out_values)))
        return ARGCSR_EINVAL;
    int4 *gi = reinterpret_cast<int4 *>(d_groupInfo);
    const size_t es = dtype_size(dtype);
#define FILL(GG, VT)                                                                              \
    Kernels<GG>::template run_fill<VT>(h.n_groups, numTiles, V, n_cols, tileGroupBase, tileSlotBase, \
                                       gscratch, d_rowPointers, d_columns, d_values,               \
                                       d_threadsMapping, gi, d_out_columns, d_out_values, tot, s)
    if (es == 8) st = G == 32 ? FILL(32, double) : G == 64 ? FILL(64, double) : FILL(128, double);
    else if (es == 4) st = G == 32 ? FILL(32, float) : G == 64 ? FILL(64, float) : FILL(128, float);
    else st = G == 32 ? FILL(32, uint16_t) : G == 64 ? FILL(64, uint16_t) : FILL(128, uint16_t);
#undef FILL
    if (st != ARGCSR_OK) return st;
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda(e, "argcsr_convert_noalloc: read status");
    if (h.status & kBadColumn) return ARGCSR_EINVAL;
    return ARGCSR_OK;
}
