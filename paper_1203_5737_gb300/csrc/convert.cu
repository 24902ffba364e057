// CSR -> ARG-CSR conversion (Section 3 of Heller & Oberhuber), every step in
// device kernels.
//
// The paper's grouping is a sequential scan: read rows in order, close the
// group after the row that takes its nonzero count above D*G, or before a row
// would become its (G+1)-th.  It is made parallel here without changing its
// result:
//   1. next[s] -- where a group that started at row s would end -- depends
//      only on s, and next[s] - s is in [1, G] (binary search in a shared
//      copy of rowPointers);
//   2. the true group starts are the chain 0, next[0], next[next[0]], ...
//      Rows are cut into tiles of T rows; since consecutive starts are at
//      most G apart, the chain enters a tile at one of its first G rows.  Per
//      tile and per possible entry, k_tile_prepare (which also computes step
//      1) finds where the chain leaves the tile and how many starts it meets
//      -- a function on G values -- by composing the same functions of
//      sub-tiles of 64 (or G) rows, whose short walks run in parallel;
//   3. k_resolve composes those functions in tile order (one CTA), which
//      gives every tile its true entry row and the index of its first group;
//   4. k_groups walks each tile from its true entry (sub-tile tables again,
//      so the walk is S short parallel walks), and for every group
//      computes the chunk size, the per-row thread counts and the group-local
//      inclusive prefix (threadsMapping), and the group's slot offset inside
//      the tile;
//   5. k_tile_scan turns the per-tile slot totals into tile offsets;
//   6. after one read-back of the totals, k_order writes the group records
//      in execution order and lists the long groups for the product, while
//      k_fill copies the CSR entries chunk by chunk into the interleaved
//      arrays; a second read-back returns the column check.
//
// Chunk size (Section 3, step 2).  The greedy -- repeatedly hand one more
// thread to the row whose chunks are fullest, until the G threads are used
// -- ends with the smallest C for which sum over rows of max(1,
// ceil(len/C)) <= G: every
// greedy step only splits a row whose filling is above that C, so it never
// overshoots, and it cannot stop above it because then the rows at the
// maximum would need fewer threads than they hold.  k_groups finds that C
// with one thread per group: from a lower bound it gallops upwards (for
// small D, where the answer is usually at or just above the bound) or
// bisects, the thread count at each trial C summed over the group's rows.
// Each row then keeps max(1,
// ceil(len/C)) threads; threads left over stay free (in the Fig. 3 example
// the last row takes four threads and one of the twelve is left over).
#include <stdio.h>

#include <mutex>
#include <type_traits>
#include <vector>

#include "internal.cuh"

namespace argcsr {
namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ void flag(unsigned *status, unsigned bits) { atomicOr(status, bits); }

// Copy delta[base, base + lim) into shared memory with 16-byte loads.  The
// delta buffer is padded to 256 bytes, so the rounded-up tail stays inside.
__device__ __forceinline__ void load_tile_delta(uint8_t *d, const uint8_t *__restrict__ delta,
                                                long long base, int lim) {
    const uint4 *src = reinterpret_cast<const uint4 *>(delta + base);
    uint4 *dst = reinterpret_cast<uint4 *>(d);
    const int n16 = (lim + 15) >> 4;
    for (int i = threadIdx.x; i < n16; i += blockDim.x) dst[i] = src[i];
}

// Sub-tiles of B rows (B >= G) cut a tile's chain walk into short pieces.
// For sub-tile s and entry e < G (the chain enters a sub-tile within its
// first G rows), fnA[s*G+e] is where the chain from row s*B+e leaves the
// sub-tile (offset past its end, < G) and cntA[s*G+e] how many group starts
// it meets.  All S*G short walks run in parallel.
template <int G>
__device__ __forceinline__ void subtile_tables(const uint8_t *d, int lim, int B, int S,
                                               uint8_t *fnA, uint8_t *cntA) {
    for (int j = threadIdx.x; j < S * G; j += blockDim.x) {
        const int sub = j / G, e = j - sub * G;
        const int end = min((sub + 1) * B, lim);
        int pos = sub * B + e, c = 0;
        while (pos < end) { ++c; pos += d[pos]; }
        fnA[j] = (uint8_t)min(max(pos - (sub + 1) * B, 0), G - 1);  // clamped past lim
        cntA[j] = (uint8_t)c;
    }
}

template <int G> constexpr int subtile_rows() { return G > 64 ? G : 64; }

// k_groups keeps per-row values (lengths, threadsMapping) in shared memory
// with one padding word after every 32: a thread per group walks its rows,
// and groups that start 32 rows apart would otherwise all hit one bank.
__host__ __device__ constexpr int pad32(int r) { return r + (r >> 5); }
__host__ __device__ constexpr size_t padded_rows(int T, int G) { return (size_t)pad32(T + G) + 1; }

// Byte offset of k_groups' threadsMapping staging array in its shared memory
// (after the parts listed at groups_smem, 4-byte aligned).
__host__ __device__ constexpr size_t groups_pfx_offset(int T, int G) {
    return ((size_t)T * 7 + 4 * padded_rows(T, G) + 2 * (size_t)(T / (G > 64 ? G : 64)) * G +
            4 * (size_t)(T / (G > 64 ? G : 64)) + 3) & ~size_t(3);
}

constexpr int kTileThreads = 512;   // threads of the per-tile kernels

// Groups are stored in execution order: by chunk size, largest first.  The
// product gives a block 8 (G = 32) groups and a block stays resident until
// its slowest group is done; in row order the largest chunk size of 8
// neighbouring groups is about 1.5 times their mean on uneven rows, so a
// third of the warp slots would sit idle.  Bucket of a chunk size: itself up
// to kLongChunk, one bucket above (long groups, any order among themselves).
constexpr int kOrderBuckets = kLongChunk + 2;
__device__ __forceinline__ int order_bucket(int C) { return C > kLongChunk ? kLongChunk + 1 : max(C, 0); }

// ---------------------------------------------------------------------------
// 1-2. Per tile: next[s] - s for every row s of the tile (and validation of
// rowPointers), then, for every entry e < G, where the chain leaves the tile
// and how many group starts it meets -- a function on G values.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kTileThreads)
k_tile_prepare(int n, long long nnz, int T, long long limit, const int *__restrict__ rp,
               uint8_t *__restrict__ delta, uint8_t *__restrict__ fn, int *__restrict__ cnt,
               DeviceTotals *tot) {
    constexpr int B = subtile_rows<G>();
    const int S = T / B;
    extern __shared__ __align__(16) uint8_t smem[];
    int *s_rp = reinterpret_cast<int *>(smem);                         // T + G + 1
    uint8_t *d = smem + 4 * ((size_t)T + G + 4);                        // T
    uint8_t *fnA = d + T;                                               // S * G
    uint8_t *cntA = fnA + (size_t)S * G;                                // S * G
    const int k = blockIdx.x;
    const long long tbase = (long long)k * T;
    const int lim = (int)min((long long)T, (long long)n - tbase);
    const int nrp = (int)min((long long)T + G + 1, (long long)n + 1 - tbase);
#pragma unroll 4
    for (int i = threadIdx.x; i < nrp; i += blockDim.x) s_rp[i] = rp[tbase + i];
    __syncthreads();
    bool bad = false;
    for (int i = threadIdx.x; i < lim; i += blockDim.x) {
        const long long sr = tbase + i;
        const int a = s_rp[i], b = s_rp[i + 1];
        bad |= (b < a) | (sr == 0 && a != 0) | (sr == n - 1 && (long long)b != nnz);
        // the group that starts at row sr ends after the first row r with
        // rp[r+1] - rp[sr] > limit, or at sr + G, or at n
        const int e = (int)min((long long)i + G, (long long)n - tbase);
        int lo = i, hi = e;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((long long)s_rp[mid + 1] - a > limit) hi = mid; else lo = mid + 1;
        }
        const int next = lo < e ? lo + 1 : e;
        d[i] = (uint8_t)(next - i);
        delta[sr] = (uint8_t)(next - i);
    }
    if (bad) flag(&tot->status, kBadRowPointers);
    __syncthreads();
    subtile_tables<G>(d, lim, B, S, fnA, cntA);
    __syncthreads();
    // compose the sub-tile functions for every entry into the tile
    for (int e = threadIdx.x; e < G; e += blockDim.x) {
        int pos = e, c = 0;
        for (int sub = 0; sub < S; ++sub) {
            c += cntA[sub * G + pos];
            pos = fnA[sub * G + pos];
        }
        fn[(size_t)k * G + e] = lim == T ? (uint8_t)pos : (uint8_t)0;
        cnt[(size_t)k * G + e] = c;
    }
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
    pdl_trigger();   // k_groups may start its per-tile work that needs no entry
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
    // the tables do not depend on the walk: load a batch of them at once
    constexpr int P = 8 / E;
    for (int kb = k0; kb < k1; kb += P) {
        int f[P][E], c[P][E];
#pragma unroll
        for (int u = 0; u < P; ++u)
            if (kb + u < k1) load_table<G>(kb + u, lane, fn, cnt, f[u], c[u]);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            if (kb + u >= k1) break;
#pragma unroll
            for (int q = 0; q < E; ++q) {
                int fp, cp;
                lookup<G>(f[u], c[u], pos[q], fp, cp);
                acc[q] += cp;
                pos[q] = fp;
            }
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
    for (int kb = k0; kb < k1; kb += P) {
        int f[P][E], c[P][E];
#pragma unroll
        for (int u = 0; u < P; ++u)
            if (kb + u < k1) load_table<G>(kb + u, lane, fn, cnt, f[u], c[u]);
#pragma unroll
        for (int u = 0; u < P; ++u) {
            if (kb + u >= k1) break;
            if (lane == 0) { tileEntry[kb + u] = entry; tileGroupBase[kb + u] = base; }
            int fp, cp;
            lookup<G>(f[u], c[u], entry, fp, cp);
            base += cp;
            entry = fp;
        }
    }
}

// ceil(l / d) for 0 <= l < 2^31 and 1 <= d < 2^31, given m = floor((2^32-1)/d):
// q = umulhi(l, m) is at most 2 below floor(l / d), so two corrections make
// it exact.  One hardware divide per divisor instead of one per row.
__device__ __forceinline__ unsigned ceil_div_by(unsigned l, unsigned d, unsigned m) {
    unsigned q = __umulhi(l, m);
    unsigned r = l - q * d;
    if (r >= d) { ++q; r -= d; }
    if (r >= d) { ++q; r -= d; }
    return q + (r != 0u);
}

// ---------------------------------------------------------------------------
// 4. Groups of a tile: chunk size, threadsMapping, slot offset in the tile.
// ---------------------------------------------------------------------------
template <int G>
__global__ void __launch_bounds__(kTileThreads)
k_groups(int n, int T, int V, int onePerRow, int gallop, const int *__restrict__ rp, const uint8_t *__restrict__ delta,
         const int *__restrict__ tileEntry, const int *__restrict__ tileGroupBase,
         int4 *__restrict__ gscratch, int *__restrict__ threadsMapping,
         long long *__restrict__ tileSlots, int *__restrict__ hist, DeviceTotals *tot) {
    constexpr int B = subtile_rows<G>();
    const int S = T / B;
    extern __shared__ __align__(16) uint8_t smem[];
    uint8_t *d = smem;                                              // T bytes
    uint16_t *starts = reinterpret_cast<uint16_t *>(smem + T);      // T entries
    int *chunk = reinterpret_cast<int *>(smem + 3 * (size_t)T);     // T entries
    int *lens = reinterpret_cast<int *>(smem + 7 * (size_t)T);      // T + G entries, padded
    uint8_t *fnA = smem + 7 * (size_t)T + 4 * padded_rows(T, G);    // S * G
    uint8_t *cntA = fnA + (size_t)S * G;                            // S * G
    uint16_t *subEntry = reinterpret_cast<uint16_t *>(cntA + (size_t)S * G);  // S
    uint16_t *subBase = subEntry + S;                                         // S
    int *pfx = reinterpret_cast<int *>(smem + groups_pfx_offset(T, G));       // T + G, padded
    __shared__ int s_count;
    __shared__ long long s_warp[kTileThreads / 32];
    __shared__ int s_hist[kOrderBuckets];
    for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_hist[i] = 0;

    const int k = blockIdx.x;
    const long long tbase = (long long)k * T;
    const int lim = (int)min((long long)T, (long long)n - tbase);
    // row lengths of the tile and of the G rows after it (a group that starts
    // in the tile may end in the next); a decreasing rowPointers is flagged in
    // k_tile_prepare, here it only has to stay bounded
    const int nl = (int)min((long long)T + G, (long long)n - tbase);
#pragma unroll 8
    for (int i = threadIdx.x; i < nl; i += blockDim.x) {
        const int a = rp[tbase + i], b = rp[tbase + i + 1];
        lens[pad32(i)] = b > a ? b - a : 0;
    }
    load_tile_delta(d, delta, tbase, lim);
    __syncthreads();
    // the chain through the tile from its true entry, in three parallel steps:
    // per sub-tile tables, one pass over the S sub-tiles, per sub-tile walks
    subtile_tables<G>(d, lim, B, S, fnA, cntA);
    __syncthreads();
    // everything above reads only rowPointers and k_tile_prepare's deltas;
    // the tile's entry and first group index come from k_resolve
    pdl_wait();
    if (threadIdx.x == 0) {
        int entry = tileEntry[k], base = 0;
        for (int sub = 0; sub < S; ++sub) {
            subEntry[sub] = (uint16_t)entry;
            subBase[sub] = (uint16_t)base;
            base += cntA[sub * G + entry];
            entry = fnA[sub * G + entry];
        }
        s_count = base;
    }
    __syncthreads();
    for (int sub = threadIdx.x; sub < S; sub += blockDim.x) {
        const int end = min((sub + 1) * B, lim);
        int pos = sub * B + subEntry[sub], c = subBase[sub];
        while (pos < end) { starts[c++] = (uint16_t)pos; pos += d[pos]; }
    }
    __syncthreads();
    const int count = s_count;
    const int gbase = tileGroupBase[k];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // one thread per group: a tile holds hundreds of groups of <= G rows
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
        const int start = starts[i];
        const int size = d[start];
        auto L = [&](int r) { return lens[pad32(start + r)]; };
        unsigned maxlen = 0;
        long long nnz = 0;
        for (int r = 0; r < size; ++r) {
            const int l = L(r);
            maxlen = max(maxlen, (unsigned)l);
            nnz += l;
        }
        long long C = 0;
        if (maxlen > 0 && onePerRow) {
            // no thread assignment: every row keeps one thread, so C is the
            // longest row -- the state the greedy starts from (Sliced
            // ELLPACK / Row-grouped CSR, Section 2)
            C = ((long long)maxlen + V - 1) / V * V;
        } else if (maxlen > 0) {
            // C >= nnz / G (all threads busy) and C >= maxlen / (G - size + 1)
            // (the longest row gets at most the spare threads plus its own)
            unsigned lo = (unsigned)max((nnz + G - 1) / G,
                                        (long long)((maxlen + (G - size)) / (G - size + 1)));
            // C = maxlen is feasible, and so is every C >= nnz / (G - size)
            // when size < G: a row keeps max(1, ceil(len/C)) < len/C + 1
            // threads, so the group needs fewer than nnz/C + size <= G
            unsigned hi = maxlen;
            if (size < G) hi = min(hi, (unsigned)((nnz + (G - size) - 1) / (G - size)));
            lo = max(lo, 1u);
            // every trial size is at least lo, so only rows longer than lo
            // can take more than one thread: when bisecting, list them once
            // (a bit per row) and visit only those in each trial
            constexpr int NW = G / 32;
            unsigned longRows[NW];
#pragma unroll
            for (int q = 0; q < NW; ++q) {
                unsigned bits = 0;
                if (!gallop) {   // uniform over the launch
                    const int r1 = min(size, 32 * (q + 1));
                    for (int r = 32 * q; r < r1; ++r) bits |= ((unsigned)L(r) > lo ? 1u : 0u) << (r - 32 * q);
                }
                longRows[q] = bits;
            }
            // threads needed with chunk size c >= lo (stops once above G)
            auto need = [&](unsigned c) {
                const unsigned m = 0xffffffffu / c;
                int t = 0;
                if (gallop) {
                    for (int r = 0; r < size && t <= G; ++r) {
                        const unsigned l = (unsigned)L(r);
                        t += l > c ? (int)ceil_div_by(l, c, m) : 1;
                    }
                    return t;
                }
                t = size;   // one thread per row, plus the extra ones of long rows
#pragma unroll
                for (int q = 0; q < NW; ++q) {
                    unsigned bits = longRows[q];
                    while (bits && t <= G) {
                        const int r = 32 * q + __ffs(bits) - 1;
                        bits &= bits - 1;
                        const unsigned l = (unsigned)L(r);
                        if (l > c) t += (int)ceil_div_by(l, c, m) - 1;
                    }
                }
                return t;
            };
            // hi is feasible.  When groups hold
            // few nonzeros (small D) the answer is usually the lower bound or
            // just above it: probe lo, lo + 1, lo + 2, lo + 4, ... until
            // feasible, then bisect the last gap.  Otherwise bisect from the
            // start.  (The choice is per launch, so a warp never runs both.)
            if (gallop && lo < hi) {
                unsigned step = 1, below = lo - 1;   // below: largest size known infeasible
                unsigned c = lo;
                while (c < hi && need(c) > G) {
                    below = c;
                    c = (hi - lo > step) ? lo + step : hi;
                    step <<= 1;
                }
                lo = below + 1;
                hi = c;
            }
            while (lo < hi) {
                const unsigned mid = lo + ((hi - lo) >> 1);
                if (need(mid) <= G) hi = mid; else lo = mid + 1;
            }
            C = ((long long)lo + V - 1) / V * V;
        }
        // thread counts and the group-local inclusive prefix (threadsMapping)
        int prefix = 0;
        const int first = (int)(tbase + start);
        const unsigned Cu = C > 0 && C <= 0x7fffffffLL ? (unsigned)C : 0u;
        const unsigned Cm = Cu ? 0xffffffffu / Cu : 0u;
        for (int r = 0; r < size; ++r) {
            const unsigned l = (unsigned)L(r);
            prefix += (Cu == 0u || l <= Cu) ? 1 : (int)ceil_div_by(l, Cu, Cm);
            pfx[pad32(start + r)] = prefix;   // copied out below with coalesced stores
        }
        // the record keeps the tile index beside the size (size <= 128)
        gscratch[gbase + i] = make_int4(first, size | (k << 8), 0, C <= 0x7fffffffLL ? (int)C : -1);
        chunk[i] = C <= 0x7fffffffLL ? (int)C : 0x7fffffff;
        if (C > 0x7fffffffLL) flag(&tot->status, kSlotOverflow);
        if (hist) atomicAdd(&s_hist[order_bucket(C <= 0x7fffffffLL ? (int)C : 0x7fffffff)], 1);
    }
    __syncthreads();
    if (hist)
        for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
            if (s_hist[i]) atomicAdd(hist + i, s_hist[i]);
    // threadsMapping of the rows this tile's groups cover: from the first
    // start to the end of the last group (which may reach into the next tile)
    if (count > 0) {
        const int rowBegin = starts[0];
        const int rowEnd = starts[count - 1] + d[starts[count - 1]];
        for (int r = rowBegin + (int)threadIdx.x; r < rowEnd; r += blockDim.x)
            threadsMapping[tbase + r] = pfx[pad32(r)];
    }
    // exclusive scan of chunk[i] * G -> slot offset of each group in the tile
    const int per = (count + kTileThreads - 1) / kTileThreads;
    const int i0 = min(count, (int)threadIdx.x * per), i1 = min(count, i0 + per);
    long long mine = 0;
    for (int i = i0; i < i1; ++i) mine += (long long)chunk[i] * G;
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
        run += (long long)chunk[i] * G;
    }
    if (threadIdx.x == kTileThreads - 1) {
        long long total = 0;
        for (int v = 0; v < kTileThreads / 32; ++v) total += s_warp[v];
        tileSlots[k] = total;
    }
}

// ---------------------------------------------------------------------------
// 5. Tile slot totals -> tile offsets; total slots.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024)
k_tile_scan(int numTiles, const long long *__restrict__ tileSlots, long long *__restrict__ tileSlotBase,
            const int *__restrict__ hist, int *__restrict__ orderBase, DeviceTotals *tot) {
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
    // first position of each chunk-size bucket in the execution order
    // (largest chunk size first): an exclusive scan by the first warp
    if (hist && warp == 0) {   // warp-uniform
        constexpr int PER = (kOrderBuckets + 31) / 32;
        int v[PER], cnt = 0;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = lane * PER + u;   // position in execution order
            v[u] = e < kOrderBuckets ? hist[kOrderBuckets - 1 - e] : 0;
            cnt += v[u];
        }
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(FULL, inc, o);
            if (lane >= o) inc += t;
        }
        int at = inc - cnt;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = lane * PER + u;
            if (e < kOrderBuckets) orderBase[kOrderBuckets - 1 - e] = at;
            at += v[u];
        }
    }
}

// ---------------------------------------------------------------------------
// 6. Group records and the chunk-wise copy (one warp per group).
// ---------------------------------------------------------------------------

// FP64 -> BF16 with one rounding to nearest even.  Going through FP32 with
// two nearest roundings can land on a BF16 tie the FP64 value was not on
// (then the tie goes to even, possibly the wrong way).  Rounding to FP32
// towards zero and setting the last bit when that was inexact ("round to
// odd", Boldo and Melquiond 2008) keeps the information a second rounding
// needs: with 24 bits against BF16's 8, the RNE of the result to BF16 equals
// the RNE of the FP64 value.  Out of FP32 range the truncation saturates at
// the largest finite FP32 value, which rounds to infinity in BF16, as the
// FP64 value does.
__device__ __forceinline__ uint16_t bf16_from_double(double v) {
    float f = __double2float_rz(v);
    if ((double)f != v && v == v) f = __uint_as_float(__float_as_uint(f) | 1u);
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// A value of the input type in the storage type: a bit copy when the two
// are the same; otherwise rounded to nearest even (BF16 is kept as its raw
// 16 bits).
template <typename VO, typename VI>
__device__ __forceinline__ VO to_storage(VI v) {
    if constexpr (std::is_same<VO, VI>::value) return v;
    else if constexpr (std::is_same<VO, float>::value && std::is_same<VI, double>::value)
        return __double2float_rn(v);
    else if constexpr (std::is_same<VO, uint16_t>::value && std::is_same<VI, double>::value)
        return bf16_from_double(v);
    else {
        static_assert(std::is_same<VO, uint16_t>::value && std::is_same<VI, float>::value,
                      "unsupported value conversion");
        return __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
}

// V consecutive elements stored with one vector store (the address is a
// multiple of V elements).
template <int V, typename T>
__device__ __forceinline__ void store_vec(T *__restrict__ p, const T (&v)[V]) {
    constexpr int B = V * (int)sizeof(T);
    if constexpr (V == 1) {
        *p = v[0];
    } else if constexpr (B == 4) {
        unsigned u;
        memcpy(&u, v, 4);
        *reinterpret_cast<unsigned *>(p) = u;
    } else if constexpr (B == 8) {
        uint2 u;
        memcpy(&u, v, 8);
        *reinterpret_cast<uint2 *>(p) = u;
    } else if constexpr (B == 16) {
        uint4 u;
        memcpy(&u, v, 16);
        *reinterpret_cast<uint4 *>(p) = u;
    } else {
        static_assert(B == 32, "unsupported vector store");
        uint4 u[2];
        memcpy(u, v, 32);
        reinterpret_cast<uint4 *>(p)[0] = u[0];
        reinterpret_cast<uint4 *>(p)[1] = u[1];
    }
}

// One chunk of a group: C elements from src (fill of them real, the rest
// padding) to slots out[(j / V) G V + j % V], j < C.
template <int G, int V, typename VT, typename VO>
__device__ __forceinline__ void copy_chunk(const int *__restrict__ cIn, const VT *__restrict__ vIn, int fill,
                                           int C, int n_cols, int *__restrict__ cOut, VO *__restrict__ vOut,
                                           bool &bad) {
    // elements per round: 8 for V >= 2 (fewer dependent load rounds per
    // chunk), 4 for V = 1, where 8 was slower at D 4 and D 8
    constexpr int R = V >= 2 ? 8 : 4;
    for (int j0 = 0; j0 < C; j0 += R) {
        int cc[R];
        VT vv[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int j = j0 + u;
            cc[u] = -1;
            memset(&vv[u], 0, sizeof(VT));
            if (j < fill) {
                cc[u] = cIn[j];
                vv[u] = vIn[j];
                bad |= (cc[u] < 0) | (cc[u] >= n_cols);
            }
        }
        // the V slots of one slot-row step sit side by side: one store each
        // (C is a multiple of V, so a step is all in or all out)
#pragma unroll
        for (int u = 0; u < R; u += V) {
            const int j = j0 + u;
            if (j < C) {
                int oc[V];
                VO ov[V];
#pragma unroll
                for (int k = 0; k < V; ++k) { oc[k] = cc[u + k]; ov[k] = to_storage<VO>(vv[u + k]); }
                const int at = (j / V) * (G * V);
                store_vec<V>(cOut + at, oc);
                store_vec<V>(vOut + at, ov);
            }
        }
    }
}

// G = 32: one warp per group (the group records are written by k_order).
// A group's loads form two dependent rounds:
// its slot base, threadsMapping words and row pointers (lane l reads those
// of row l; the bounds of the row a chunk belongs to come by shuffle), then
// its entries.  The record of the warp's next group is loaded one group
// ahead.
template <typename VT, typename VO, int V>
__device__ __forceinline__ void fill_g32(long long nGroups, int n_cols, const long long *__restrict__ tileSlotBase,
                                         const int4 *__restrict__ gscratch, const int *__restrict__ rp,
                                         const int *__restrict__ colsIn, const VT *__restrict__ valsIn,
                                         const int *__restrict__ threadsMapping, int4 *__restrict__ groupInfo,
                                         int *__restrict__ colsOut, VO *__restrict__ valsOut,
                                         DeviceTotals *tot) {
    const int lane = threadIdx.x & 31;
    const long long W = (long long)gridDim.x * (blockDim.x >> 5);
    long long t = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    bool bad = false;
    // groups in descending order: the product that follows a conversion
    // reads them in ascending order and finds the last ones written (the
    // first groups) still in L2
    int4 next = t < nGroups ? gscratch[nGroups - 1 - t] : make_int4(0, 0, 0, 0);
    for (; t < nGroups; t += W) {
        const long long g = nGroups - 1 - t;
        const int4 s = next;
        if (t + W < nGroups) next = gscratch[g - W];
        const int first = s.x, size = s.y & 255, C = s.w;
        const int off = (int)(tileSlotBase[s.y >> 8] + s.z);
        const int end = lane < size ? threadsMapping[first + lane] : 0;
        const int rowStart = lane < size ? rp[first + lane] : 0;
        const int lastEnd = rp[first + size];
        if (C <= 0) continue;   // warp-uniform
        // row ends as a bit mask: the row of chunk `lane` is the number of
        // ends below it, its first chunk follows the previous end
        const unsigned ends = __reduce_or_sync(FULL, lane < size ? 1u << (end - 1) : 0u);
        const unsigned below = ends & ((1u << lane) - 1u);
        const int row = __popc(below), begin = below ? 32 - __clz(below) : 0;
        const int rs = __shfl_sync(FULL, rowStart, min(row, 31));
        const int reNext = __shfl_sync(FULL, rowStart, min(row + 1, 31));
        int src = 0, fill = 0;
        if (row < size) {
            const int re = row + 1 < size ? reNext : lastEnd;
            src = rs + (lane - begin) * C;
            fill = max(0, min(C, re - src));
        }
        copy_chunk<32, V>(colsIn + src, valsIn + src, fill, C, n_cols, colsOut + off + lane * V,
                          valsOut + off + lane * V, bad);
    }
    if (__any_sync(FULL, bad) && lane == 0) flag(&tot->status, kBadColumn);
}

template <int G, typename VT, typename VO, int V>
__global__ void __launch_bounds__(256)
k_fill(long long nGroups, int n_cols, const long long *__restrict__ tileSlotBase,
       const int4 *__restrict__ gscratch, const int *__restrict__ rp, const int *__restrict__ colsIn,
       const VT *__restrict__ valsIn, const int *__restrict__ threadsMapping,
       int4 *__restrict__ groupInfo, int *__restrict__ colsOut, VO *__restrict__ valsOut,
       DeviceTotals *tot) {
    if constexpr (G == 32) {
        fill_g32<VT, VO, V>(nGroups, n_cols, tileSlotBase, gscratch, rp, colsIn, valsIn, threadsMapping,
                            groupInfo, colsOut, valsOut, tot);
        pdl_wait();   // this kernel ends after k_order, which runs alongside it
    } else {
        // G = 64 or 128: one group per warp; the row of each chunk from a
        // per-warp table built from threadsMapping
        __shared__ short s_rowOf[8][G];
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
        bool bad = false;
        for (long long g = (long long)blockIdx.x * (blockDim.x >> 5) + warp; g < nGroups; g += warps) {
            const int4 s = gscratch[g];
            const int first = s.x, size = s.y & 255, C = s.w;
            const long long off = tileSlotBase[s.y >> 8] + s.z;
            if (C <= 0) continue;
            for (int c = lane; c < G; c += 32) s_rowOf[warp][c] = -1;
            __syncwarp();
            for (int r = lane; r < size; r += 32) {
                const int b = r ? threadsMapping[first + r - 1] : 0, e = threadsMapping[first + r];
                for (int c = b; c < e; ++c) s_rowOf[warp][c] = (short)r;
            }
            __syncwarp();
#pragma unroll
            for (int q = 0; q < G / 32; ++q) {
                const int c = q * 32 + lane;
                int row = s_rowOf[warp][c];
                if (row < 0) row = size;
                const int begin = (row > 0 && row < size) ? threadsMapping[first + row - 1] : 0;
                int src = 0, fill = 0;
                if (row < size) {
                    const int rs = rp[first + row], re = rp[first + row + 1];
                    src = rs + (c - begin) * C;
                    fill = max(0, min(C, re - src));
                }
                // a chunk's elements are contiguous in the CSR arrays; lanes of
                // one row read C apart, which L1 serves from the lines already
                // fetched
                copy_chunk<G, V>(colsIn + src, valsIn + src, fill, C, n_cols, colsOut + off + c * V,
                                 valsOut + off + c * V, bad);
            }
            __syncwarp();
        }
        if (__any_sync(FULL, bad) && lane == 0) flag(&tot->status, kBadColumn);
        pdl_wait();   // this kernel ends after k_order, which runs alongside it
    }
}

// The group records (Listing 1) from the structure pass, one thread per
// group: its slot offset completed with its tile's base, placed in
// execution order (largest chunk size first; orderCursor holds each
// sub-bucket's first position and hands positions out) or, without
// orderCursor, in row order.  The long groups (G = 32, V = 1) are listed by
// their position for the product.
__global__ void __launch_bounds__(256)
k_order(long long nGroups, const long long *__restrict__ tileSlotBase, const int4 *__restrict__ gscratch,
        int4 *__restrict__ groupInfo, int *__restrict__ orderCursor, int *__restrict__ longList,
        long long longCap, DeviceTotals *tot) {
    pdl_trigger();   // k_fill reads nothing this kernel writes: it may run alongside
    // positions are handed out per block: ranks inside the block from
    // shared-memory counters, then one global reservation per bucket the
    // block uses
    __shared__ int s_cnt[kOrderBuckets], s_base[kOrderBuckets];
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = g < nGroups;
    const int4 s = on ? gscratch[g] : make_int4(0, 0, 0, 0);
    const int size = s.y & 255, C = s.w;
    long long pos = g;
    if (orderCursor) {   // block-uniform
        for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) s_cnt[i] = 0;
        __syncthreads();
        const int b = order_bucket(C);
        const int r = on ? atomicAdd(&s_cnt[b], 1) : 0;
        __syncthreads();
        for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x)
            if (s_cnt[i]) s_base[i] = atomicAdd(orderCursor + i, s_cnt[i]);
        __syncthreads();
        pos = s_base[b] + r;
    }
    if (!on) return;
    const int off = (int)(tileSlotBase[s.y >> 8] + s.z);
    groupInfo[pos] = make_int4(s.x, size, off, C);
    if (longList && C > kLongChunk) {
        const long long i = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&tot->n_long), 1ull);
        if (i < longCap) longList[i] = (int)pos;
    }
}

// Dynamic shared memory of k_groups: delta (T), starts (2T), chunk sizes
// (4T), row lengths (4(T+G), padded), sub-tile tables (2 S G), sub-tile
// entries and bases (4 S), threadsMapping of the tile's rows (4(T+G), padded).
inline size_t groups_smem(int T, int G) {
    const int S = T / (G > 64 ? G : 64);
    (void)S;
    return groups_pfx_offset(T, G) + 4 * padded_rows(T, G);
}
// Dynamic shared memory of k_tile_prepare: rowPointers (4(T+G+4)), delta
// (T), sub-tile tables (2 S G).
inline size_t prepare_smem(int T, int G) {
    const int S = T / (G > 64 ? G : 64);
    return 4 * ((size_t)T + G + 4) + (size_t)T + 2 * (size_t)S * G;
}

// Kernels for one group size.
template <int G>
struct Kernels {
    static argcsr_status run_structure(int n, long long nnz, long long limit, int T, int numTiles,
                                       int V, int onePerRow, const int *rp, uint8_t *delta, uint8_t *fn, int *cnt,
                                       int *tileEntry, int *tileGroupBase, int4 *gscratch, int *tm,
                                       long long *tileSlots, long long *tileSlotBase, int *hist,
                                       int *orderBase, DeviceTotals *tot, cudaStream_t s) {
        {
            TraceScope t("k_tile_prepare", s);
            k_tile_prepare<G><<<numTiles, kTileThreads, prepare_smem(T, G), s>>>(n, nnz, T, limit, rp, delta,
                                                                       fn, cnt, tot);
        }
        {
            TraceScope t("k_resolve", s);
            k_resolve<G><<<1, 1024, 0, s>>>(numTiles, fn, cnt, tileEntry, tileGroupBase, tot);
        }
        {
            TraceScope t("k_groups", s);
            const size_t smem = groups_smem(T, G);
            // launched behind k_resolve's start: the per-tile work that needs
            // no tile entry overlaps k_resolve's single block
            const cudaError_t e = launch_pdl(k_groups<G>, (unsigned)numTiles, kTileThreads, smem, s, n, T, V, onePerRow,
                                             limit <= 6LL * G ? 1 : 0, rp, (const uint8_t *)delta,
                                             (const int *)tileEntry, (const int *)tileGroupBase, gscratch, tm,
                                             tileSlots, hist, tot);
            if (e != cudaSuccess) return record_cuda(e, "k_groups launch");
        }
        {
            TraceScope t("k_tile_scan", s);
            k_tile_scan<<<1, 1024, 0, s>>>(numTiles, tileSlots, tileSlotBase, hist, orderBase, tot);
        }
        count_launches(4);
        ARGCSR_CHECK_LAUNCH("conversion structure kernels");
        return ARGCSR_OK;
    }
    template <typename VT, typename VO = VT>
    static argcsr_status run_fill(long long nGroups, int V, int n_cols,
                                  const long long *tileSlotBase,
                                  const int4 *gscratch, const int *rp, const int *cols,
                                  const void *vals, const int *tm, int4 *gi, int *colsOut,
                                  void *valsOut, int *longList, long long longCap, int *orderCursor,
                                  DeviceTotals *tot, cudaStream_t s) {
        if (nGroups == 0) return ARGCSR_OK;
        {
            TraceScope t("k_order", s);
            k_order<<<(unsigned)((nGroups + 255) / 256), 256, 0, s>>>(nGroups, tileSlotBase, gscratch, gi,
                                                                    orderCursor, longList, longCap, tot);
            count_launches(1);
        }
        const long long blocks = min((nGroups + 7) / 8, 152LL * 64);
        TraceScope t("k_fill", s);
        const VT *v = static_cast<const VT *>(vals);
        VO *vo = static_cast<VO *>(valsOut);
        // launched behind k_order's start (programmatic serialization): the
        // two share no data, and k_fill's last act waits for k_order
        cudaError_t e;
        if (V == 1)
            e = launch_pdl(k_fill<G, VT, VO, 1>, (unsigned)blocks, 256, 0, s, nGroups, n_cols,
                           (const long long *)tileSlotBase, (const int4 *)gscratch, rp, cols, v, tm, gi, colsOut,
                           vo, tot);
        else if (V == 2)
            e = launch_pdl(k_fill<G, VT, VO, 2>, (unsigned)blocks, 256, 0, s, nGroups, n_cols,
                           (const long long *)tileSlotBase, (const int4 *)gscratch, rp, cols, v, tm, gi, colsOut,
                           vo, tot);
        else
            e = launch_pdl(k_fill<G, VT, VO, 4>, (unsigned)blocks, 256, 0, s, nGroups, n_cols,
                           (const long long *)tileSlotBase, (const int4 *)gscratch, rp, cols, v, tm, gi, colsOut,
                           vo, tot);
        if (e != cudaSuccess) return record_cuda(e, "k_fill launch");
        count_launches(1);
        ARGCSR_CHECK_LAUNCH("k_fill");
        return ARGCSR_OK;
    }
};

template <int G>
argcsr_status set_smem_limits(int T) {
    cudaError_t e = cudaFuncSetAttribute(k_groups<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)groups_smem(T, G));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tile_prepare<G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)prepare_smem(T, G));
    if (e != cudaSuccess) return record_cuda(e, "cudaFuncSetAttribute");
    return ARGCSR_OK;
}

// Pinned host copies of the totals for the two status reads (a copy into
// pageable memory goes through a driver staging buffer and returns later),
// kept for reuse.
std::mutex g_totals_mu;
std::vector<DeviceTotals *> g_totals_free;

struct PinnedTotals {
    DeviceTotals *p = nullptr;
    PinnedTotals() {
        {
            std::lock_guard<std::mutex> lock(g_totals_mu);
            if (!g_totals_free.empty()) {
                p = g_totals_free.back();
                g_totals_free.pop_back();
                return;
            }
        }
        if (cudaHostAlloc((void **)&p, sizeof(DeviceTotals), cudaHostAllocDefault) != cudaSuccess) p = nullptr;
    }
    ~PinnedTotals() {
        if (!p) return;
        std::lock_guard<std::mutex> lock(g_totals_mu);
        g_totals_free.push_back(p);
    }
};

struct Scratch {
    void *p[10] = {};
    cudaStream_t s;
    ~Scratch() { for (void *q : p) pool_free(q, s); }
};

}  // namespace
}  // namespace argcsr

using namespace argcsr;

namespace {
// input -> storage value types a conversion accepts: the same type, or a
// narrowing one (f64 -> f32, f64 -> bf16, f32 -> bf16)
bool conversion_supported(argcsr_dtype in, argcsr_dtype st) {
    return in == st || (in == ARGCSR_F64 && (st == ARGCSR_F32 || st == ARGCSR_BF16)) ||
           (in == ARGCSR_F32 && st == ARGCSR_BF16);
}
}  // namespace

extern "C" ARGCSR_API argcsr_status argcsr_create_from_csr(
    int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *d_rowPointers,
    const int32_t *d_columns, const void *d_values, argcsr_dtype dtype, const argcsr_params *params,
    argcsr_stream_t stream, argcsr_t *out) {
    return argcsr_create_from_csr_as(n_rows, n_cols, nnz, d_rowPointers, d_columns, d_values, dtype,
                                     dtype, params, stream, out);
}

extern "C" ARGCSR_API argcsr_status argcsr_create_from_csr_as(
    int32_t n_rows, int32_t n_cols, int64_t nnz, const int32_t *d_rowPointers,
    const int32_t *d_columns, const void *d_values, argcsr_dtype in_dtype, argcsr_dtype dtype,
    const argcsr_params *params, argcsr_stream_t stream, argcsr_t *out) {
    if (!out) return ARGCSR_EINVAL;
    *out = nullptr;
    if (in_dtype != ARGCSR_F64 && in_dtype != ARGCSR_F32 && in_dtype != ARGCSR_BF16) return ARGCSR_EINVAL;
    if (!params || n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL) return ARGCSR_EINVAL;
    const int G = params->group_size, D = params->desired_chunk_size, V = params->vec_width;
    const int P1 = params->one_thread_per_row;
    if ((G != 32 && G != 64 && G != 128) || D < 1 || (V != 1 && V != 2 && V != 4)) return ARGCSR_EINVAL;
    if (P1 != 0 && P1 != 1) return ARGCSR_EINVAL;
    if (dtype != ARGCSR_F64 && dtype != ARGCSR_F32 && dtype != ARGCSR_BF16) return ARGCSR_EINVAL;
    if (!conversion_supported(in_dtype, dtype)) return ARGCSR_ENOTSUP;
    if (!d_rowPointers || (nnz > 0 && (!d_columns || !d_values))) return ARGCSR_EINVAL;
    if (n_rows == 0 && nnz != 0) return ARGCSR_EINVAL;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

    argcsr_matrix *A = new argcsr_matrix();
    cudaGetDevice(&A->device);
    A->n_rows = n_rows; A->n_cols = n_cols; A->nnz = nnz;
    A->G = G; A->D = D; A->V = V; A->one_per_row = P1; A->dtype = dtype;
    auto fail = [&](argcsr_status st) { argcsr_destroy(A, stream); return st; };
    if (n_rows == 0) { *out = A; return ARGCSR_OK; }

    const int n = n_rows;
    // tiles of 2048 rows give a 2M-row matrix about 1000 per-tile blocks;
    // very large matrices use longer tiles to keep k_resolve's table short
    // (8192 rows: the per-tile kernels' shared memory stays below 143 KB)
    const int T = n <= (1 << 25) ? 2048 : 8192;
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
    ALLOC(9, 2 * kOrderBuckets * sizeof(int));            // chunk-size histogram, bucket cursors
    if ((st = pool_alloc((void **)&A->d_threadsMapping, (size_t)n * 4, s)) != ARGCSR_OK) return fail(st);
#undef ALLOC
    uint8_t *delta = (uint8_t *)sc.p[0];
    uint8_t *fn = (uint8_t *)sc.p[1];
    int *cnt = (int *)sc.p[2], *tileEntry = (int *)sc.p[3], *tileGroupBase = (int *)sc.p[4];
    int4 *gscratch = (int4 *)sc.p[5];
    long long *tileSlots = (long long *)sc.p[6], *tileSlotBase = (long long *)sc.p[7];
    DeviceTotals *tot = (DeviceTotals *)sc.p[8];
    int *hist = (int *)sc.p[9], *orderBase = hist + kOrderBuckets;

    cudaError_t e = cudaMemsetAsync(tot, 0, sizeof(DeviceTotals), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, kOrderBuckets * sizeof(int), s);
    if (e != cudaSuccess) return fail(record_cuda(e, "cudaMemsetAsync"));
    A->execution_order = 1;
    const long long limit = (long long)D * G;
    switch (G) {
        case 32: st = set_smem_limits<32>(T); if (!st) st = Kernels<32>::run_structure(n, nnz, limit, T, numTiles, V, P1, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, A->d_threadsMapping, tileSlots, tileSlotBase, hist, orderBase, tot, s); break;
        case 64: st = set_smem_limits<64>(T); if (!st) st = Kernels<64>::run_structure(n, nnz, limit, T, numTiles, V, P1, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, A->d_threadsMapping, tileSlots, tileSlotBase, hist, orderBase, tot, s); break;
        default: st = set_smem_limits<128>(T); if (!st) st = Kernels<128>::run_structure(n, nnz, limit, T, numTiles, V, P1, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, A->d_threadsMapping, tileSlots, tileSlotBase, hist, orderBase, tot, s); break;
    }
    if (st != ARGCSR_OK) return fail(st);

    PinnedTotals ht;
    if (!ht.p) return fail(ARGCSR_ENOMEM);
    DeviceTotals &h = *ht.p;
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
    // k_fill lists the long groups (G = 32, V = 1) for the SpMV; a long
    // group holds more than kLongChunk * 32 slots
    const long long longCap = G == 32 && V == 1 ? A->n_slots / ((long long)kLongChunk * 32) : 0;
    if (longCap > 0 &&
        (st = pool_alloc((void **)&A->d_longGroups, (size_t)longCap * 4, s)) != ARGCSR_OK)
        return fail(st);

#define FILL(GG, VI, VO)                                                                         \
    Kernels<GG>::template run_fill<VI, VO>(A->n_groups, V, n_cols, tileSlotBase,                   \
                                           gscratch, d_rowPointers, d_columns, d_values,          \
                                           A->d_threadsMapping, A->d_groupInfo, A->d_columns,     \
                                           A->d_values, A->d_longGroups, longCap, orderBase, tot, s)
#define FILL_G(VI, VO) (G == 32 ? FILL(32, VI, VO) : G == 64 ? FILL(64, VI, VO) : FILL(128, VI, VO))
    if (in_dtype == dtype) {
        if (es == 8) st = FILL_G(double, double);
        else if (es == 4) st = FILL_G(float, float);
        else st = FILL_G(uint16_t, uint16_t);
    } else if (in_dtype == ARGCSR_F64) {
        st = dtype == ARGCSR_F32 ? FILL_G(double, float) : FILL_G(double, uint16_t);
    } else {
        st = FILL_G(float, uint16_t);
    }
#undef FILL_G
#undef FILL
    if (st != ARGCSR_OK) return fail(st);
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(record_cuda(e, "conversion: read status"));
    if (h.status & kBadColumn) return fail(ARGCSR_EINVAL);
    A->n_long = longCap > 0 ? (h.n_long < longCap ? h.n_long : longCap) : 0;
    if (A->n_long == 0 && A->d_longGroups) {
        pool_free(A->d_longGroups, s);
        A->d_longGroups = nullptr;
    }

    A->device_bytes = (int64_t)A->n_groups * 16 + (int64_t)n * 4 + A->n_slots * (4 + (int64_t)es) +
                      (A->d_longGroups ? longCap * 4 : 0);
    *out = A;
    return ARGCSR_OK;
}

// ---------------------------------------------------------------------------
// argcsr_convert_noalloc: the conversion with every intermediate array in one
// file-scope device array, for callers that must not allocate device memory.
// ---------------------------------------------------------------------------
namespace argcsr {
namespace {

constexpr int kNoallocTile = 2048;   // the tile of argcsr_create_from_csr for n <= 2^25
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
    if (dev < 0 || dev >= 64) {
        set_error_message("argcsr_convert_noalloc: device ordinal above 63");
        return ARGCSR_ENOTSUP;
    }
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
    // every failure below leaves a message for argcsr_last_error_message()
    auto fail = [](argcsr_status st, const char *why) {
        set_error_message(why);
        return st;
    };
    if (!h_n_groups || !h_n_slots) return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: null size outputs");
    *h_n_groups = 0;
    *h_n_slots = 0;
    if (!params || n_rows < 0 || n_cols < 0 || nnz < 0 || nnz > 0x7fffffffLL)
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: bad sizes or null params");
    if (n_rows > ARGCSR_NOALLOC_MAX_ROWS)
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: n_rows exceeds ARGCSR_NOALLOC_MAX_ROWS");
    const int G = params->group_size, D = params->desired_chunk_size, V = params->vec_width;
    const int P1 = params->one_thread_per_row;
    if ((G != 32 && G != 64 && G != 128) || D < 1 || (V != 1 && V != 2 && V != 4) || (P1 != 0 && P1 != 1))
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: bad group size, chunk size, vector width or mode");
    if (dtype != ARGCSR_F64 && dtype != ARGCSR_F32 && dtype != ARGCSR_BF16)
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: bad dtype");
    if (!d_rowPointers || (nnz > 0 && (!d_columns || !d_values)))
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: null input array");
    if (n_rows == 0)
        return nnz == 0 ? ARGCSR_OK : fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: nnz > 0 with no rows");
    if (!d_threadsMapping || group_capacity < 0 || slot_capacity < 0)
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: null threadsMapping or negative capacity");
    if (reinterpret_cast<uintptr_t>(d_groupInfo) % 16)   // int4 records
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: d_groupInfo is not 16-byte aligned");
    // k_fill stores the V slots of a slot-row step with one vector store
    if (V > 1 && (reinterpret_cast<uintptr_t>(d_out_columns) % 16 || reinterpret_cast<uintptr_t>(d_out_values) % 16))
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: with vec_width above 1 the output arrays must be 16-byte aligned");
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
    const long long limit = (long long)D * G;
    switch (G) {
        case 32: st = set_smem_limits<32>(T); if (!st) st = Kernels<32>::run_structure(n, nnz, limit, T, numTiles, V, P1, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, d_threadsMapping, tileSlots, tileSlotBase, nullptr, nullptr, tot, s); break;
        case 64: st = set_smem_limits<64>(T); if (!st) st = Kernels<64>::run_structure(n, nnz, limit, T, numTiles, V, P1, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, d_threadsMapping, tileSlots, tileSlotBase, nullptr, nullptr, tot, s); break;
        default: st = set_smem_limits<128>(T); if (!st) st = Kernels<128>::run_structure(n, nnz, limit, T, numTiles, V, P1, d_rowPointers, delta, fn, cnt, tileEntry, tileGroupBase, gscratch, d_threadsMapping, tileSlots, tileSlotBase, nullptr, nullptr, tot, s); break;
    }
    if (st != ARGCSR_OK) return st;
    // the totals come back into this stack copy: a copy into pageable
    // memory returns once it is done, and the synchronisation orders it in
    // any case; no pinned buffer is taken (allocating one is what this entry
    // point exists to avoid)
    DeviceTotals h{};
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda(e, "argcsr_convert_noalloc: read totals");
    if (h.status & kBadRowPointers)
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: rowPointers not monotone from 0 to nnz");
    if (h.status & kSlotOverflow)
        return fail(ARGCSR_EOVERFLOW, "argcsr_convert_noalloc: more than 2^31 - 1 slots");
    *h_n_groups = h.n_groups;
    *h_n_slots = h.n_slots;
    if (h.n_groups > group_capacity || h.n_slots > slot_capacity)
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: output capacity too small (required sizes returned)");
    if ((h.n_groups > 0 && !d_groupInfo) || (h.n_slots > 0 && (!d_out_columns || !d_out_values)))
        return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: null output array");
    int4 *gi = reinterpret_cast<int4 *>(d_groupInfo);
    const size_t es = dtype_size(dtype);
#define FILL(GG, VT)                                                                              \
    Kernels<GG>::template run_fill<VT>(h.n_groups, V, n_cols, tileSlotBase,                        \
                                       gscratch, d_rowPointers, d_columns, d_values,               \
                                       d_threadsMapping, gi, d_out_columns, d_out_values, nullptr, 0, \
                                       nullptr, tot, s)
    if (es == 8) st = G == 32 ? FILL(32, double) : G == 64 ? FILL(64, double) : FILL(128, double);
    else if (es == 4) st = G == 32 ? FILL(32, float) : G == 64 ? FILL(64, float) : FILL(128, float);
    else st = G == 32 ? FILL(32, uint16_t) : G == 64 ? FILL(64, uint16_t) : FILL(128, uint16_t);
#undef FILL
    if (st != ARGCSR_OK) return st;
    e = cudaMemcpyAsync(&h, tot, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return record_cuda(e, "argcsr_convert_noalloc: read status");
    if (h.status & kBadColumn) return fail(ARGCSR_EINVAL, "argcsr_convert_noalloc: column index out of range");
    return ARGCSR_OK;
}
