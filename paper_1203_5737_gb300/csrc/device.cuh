// Device helpers shared by the SpMV, SpMM and batched kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

namespace argcsr {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ double widen(double v) { return v; }
__device__ __forceinline__ float widen(float v) { return v; }
__device__ __forceinline__ float widen(uint16_t bits) { return __uint_as_float((unsigned)bits << 16); }

// Streaming (evict-first) loads of V consecutive elements, V*sizeof(T) in
// {2, 4, 8, 16, 32} bytes, from an address aligned to that size.
template <typename T, int V>
__device__ __forceinline__ void ld_stream(const T *p, T (&out)[V]) {
    constexpr int B = (int)sizeof(T) * V;
    if constexpr (B == 2) {
        unsigned short u = __ldcs(reinterpret_cast<const unsigned short *>(p));
        memcpy(out, &u, 2);
    } else if constexpr (B == 4) {
        unsigned u = __ldcs(reinterpret_cast<const unsigned *>(p));
        memcpy(out, &u, 4);
    } else if constexpr (B == 8) {
        uint2 u = __ldcs(reinterpret_cast<const uint2 *>(p));
        memcpy(out, &u, 8);
    } else if constexpr (B == 16) {
        uint4 u = __ldcs(reinterpret_cast<const uint4 *>(p));
        memcpy(out, &u, 16);
    } else {
        static_assert(B == 32, "unsupported vector width");
        uint4 u0 = __ldcs(reinterpret_cast<const uint4 *>(p));
        uint4 u1 = __ldcs(reinterpret_cast<const uint4 *>(p) + 1);
        memcpy(out, &u0, 16);
        memcpy(reinterpret_cast<char *>(out) + 16, &u1, 16);
    }
}

// Gather of one x element.  OP selects the load instruction: 0 the
// read-only path (ld.global.nc), 1 the read-only path without allocating in
// L1 (x lines are rarely reused there: a warp's 32 gathers hit 32 random
// lines), 2 L2 only (ld.global.cg), 3 the default caching load.
#ifndef ARGCSR_GATHER_OP
#define ARGCSR_GATHER_OP 0
#endif
template <int OP = ARGCSR_GATHER_OP>
__device__ __forceinline__ double ldx(const double *p) {
    if constexpr (OP == 0) return __ldg(p);
    double v;
    if constexpr (OP == 1) asm("ld.global.nc.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
    else if constexpr (OP == 2) asm("ld.global.cg.f64 %0, [%1];" : "=d"(v) : "l"(p));
    else asm("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
template <int OP = ARGCSR_GATHER_OP>
__device__ __forceinline__ float ldx(const float *p) {
    if constexpr (OP == 0) return __ldg(p);
    float v;
    if constexpr (OP == 1) asm("ld.global.nc.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
    else if constexpr (OP == 2) asm("ld.global.cg.f32 %0, [%1];" : "=f"(v) : "l"(p));
    else asm("ld.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

// sum += v on lanes where `on` holds.  Written as a predicated PTX add so
// that lanes without work issue no FP64 operation (a plain conditional add
// may be turned into an add on every lane followed by a select).
__device__ __forceinline__ void add_if(double &sum, double v, bool on) {
    asm("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p add.rn.f64 %0, %0, %1;\n\t}"
        : "+d"(sum) : "d"(v), "r"((unsigned)on));
}
__device__ __forceinline__ void add_if(float &sum, float v, bool on) {
    if (on) sum += v;
}

// Row of each chunk of a G = 32 group, from threadsMapping: a bit mask of
// row ends (bit k set <=> chunk k is the last chunk of a row) built with one
// warp reduction; the lane's row is the number of ends below it.
struct WarpRowMap {
    unsigned ends;      // row-end mask
    int row;            // local row of this lane's chunk (== size for free chunks)
    int segStart;       // first chunk (lane) of that row
    int segEnd;         // one past its last chunk
    bool owns;          // the lane's chunk belongs to a row
    __device__ __forceinline__ WarpRowMap(const int *__restrict__ tm, int first, int size, int lane) {
        const int end = lane < size ? __ldg(tm + first + lane) : 0;
        ends = __reduce_or_sync(FULL, lane < size ? 1u << (end - 1) : 0u);
        const unsigned below = ends & ((1u << lane) - 1u);
        row = __popc(below);
        owns = row < size;
        segStart = below ? 32 - __clz(below) : 0;
        const unsigned atOrAbove = ends & ~((1u << lane) - 1u);
        segEnd = atOrAbove ? __ffs(atOrAbove) : 0;
    }
};

}  // namespace argcsr
