// Device helpers shared by the solver kernels: GPU-scope relaxed loads and
// stores, the "not yet solved" marker, bounded dependency waits and the
// status word.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sptrsv {

// Status word: (row << 32) | code.  atomicMin keeps the lowest failing row
// (and, for one row, the lowest code).  ~0ull means "no failure".
constexpr unsigned long long kStatusClear = ~0ull;
enum : int { kCodeStructure = 2, kCodeZeroPivot = 3, kCodeTimeout = 6, kCodeInternal = 8 };

__device__ __forceinline__ void report(unsigned long long* status, int row, int code) {
    unsigned long long v = ((unsigned long long)(unsigned)row << 32) | (unsigned)code;
    atomicMin(status, v);
}

// ---------------------------------------------------------------------------
// Relaxed loads/stores at GPU scope.  A relaxed access is single-copy atomic
// for naturally aligned 4/8-byte words and is served by L2 (the coherence
// point), never by a stale L1 line.  A published value is the only datum a
// waiting row needs, so no acquire/release ordering is required.
__device__ __forceinline__ double ld_relaxed(const double* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return __longlong_as_double((long long)v);
}
__device__ __forceinline__ float ld_relaxed(const float* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return __uint_as_float(v);
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"((unsigned long long)__double_as_longlong(v)) : "memory");
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(__float_as_uint(v)) : "memory");
}
__device__ __forceinline__ void st_relaxed(int* p, int v) {
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// "Not yet solved" marker.  The self-scheduled solve fills x with all-ones
// bit patterns (a NaN; a result that happens to carry exactly this pattern
// is rewritten to the canonical quiet NaN before it is published), so a
// published value doubles as its own ready flag.
template <typename T> struct Marker;
template <> struct Marker<double> {
    static __device__ __forceinline__ bool pending(double v) {
        return (unsigned long long)__double_as_longlong(v) == ~0ull;
    }
    static __device__ __forceinline__ double pending_value() { return __longlong_as_double(-1ll); }
    static __device__ __forceinline__ double canonical_nan() {
        return __longlong_as_double(0x7ff8000000000000ll);
    }
};
template <> struct Marker<float> {
    static __device__ __forceinline__ bool pending(float v) { return __float_as_uint(v) == ~0u; }
    static __device__ __forceinline__ float pending_value() { return __uint_as_float(~0u); }
    static __device__ __forceinline__ float canonical_nan() { return __uint_as_float(0x7fc00000u); }
};

// The one bit pattern a published value must not have is the marker itself
// (an integer compare: FP64 instructions are scarce on GB300).
template <typename T>
__device__ __forceinline__ T publishable(T v) {
    return Marker<T>::pending(v) ? Marker<T>::canonical_nan() : v;
}

// Spin policy of a dependency wait: a few hot polling rounds, then rounds
// spaced by a growing __nanosleep (capped), at most `limit` rounds in one
// wait; past the limit the wait records SPTRSV_ERR_TIMEOUT for its row and
// goes on with NaN, so every later row still finishes.
struct SpinPolicy {
    long long limit;
    int hot;          // polls before the first sleep
    unsigned max_ns;  // back-off cap
};

// Entries a lane loads at once (one chunk) in the self-scheduled kernels.
constexpr int kChunk = 4;

// sum - a[0] v[0] - a[1] v[1] - ... over the live entries of a chunk, one FMA
// each in slot order (the fold order of every form: farthest dependency
// first, so a row's diagonal, stored last in fold order, is never before a
// live slot).  The dead slots of a chunk (the diagonal, past the
// row's end) lie before its first live entry (the diagonal of an upper row)
// or after its last one (the diagonal of a lower row, the row's end), and the
// loop covers only the slots in between: a predicated-off FP64 instruction
// still sits on the dependency chain of `sum` for a whole FP64 issue slot (on
// GB300 each skipped slot saved ~50 ns per dependency hop).
template <typename T, int E>
__device__ __forceinline__ T fold_chunk(T sum, const T (&a)[E], const T (&v)[E], unsigned live) {
    const int hi = 32 - __clz(live);
    const int lo = __ffs(live) - 1;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if (e >= hi) break;
        if (e < lo) continue;
        if (live & (1u << e)) sum = fma(-a[e], v[e], sum);
    }
    return sum;
}

// Mask of the W-lane group (sub-warp) that `lane` belongs to.
template <int W>
__device__ __forceinline__ unsigned group_mask(int lane) {
    if (W >= 32) return 0xffffffffu;
    return ((1u << (W & 31)) - 1u) << ((lane / W) * W);
}

template <int W, typename T>
__device__ __forceinline__ T group_sum(T v, unsigned mask) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// group_sum over the first `span` lanes of every group, the others holding
// +0.0 (warp-uniform span, 1 <= span <= W): a butterfly level whose partner
// lanes are all zero would add +0.0 and is skipped.  The result in the
// group's first lane equals group_sum's (x + 0.0 == x; only a -0.0 partial
// sum may come out as -0.0 instead of +0.0).  Each level is a dependent FP64
// add of 64 cycles on GB300, so short rows save one per halving of span.
template <int W, typename T>
__device__ __forceinline__ T group_sum_span(T v, unsigned mask, int span) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1)
        if (off < span) v += __shfl_xor_sync(mask, v, off);
    return v;
}

// Warp-uniform span of the rows a warp holds: the longest of its rows'
// stored entries, at most W (a lane at or past it holds no entry of its row).
template <int W>
__device__ __forceinline__ int warp_span(bool has_row, int len) {
    if (W == 1) return 1;
    const int l = has_row ? (len < W ? len : W) : 0;
    return (int)__reduce_max_sync(0xffffffffu, (unsigned)l);
}

template <int W>
__device__ __forceinline__ int group_max(int v, unsigned mask) {
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(mask, v, off));
    return v;
}

}  // namespace sptrsv
