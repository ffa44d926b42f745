// Column-wise self-scheduled solve (Alg. 4, SLFC), one right-hand side.
//
// The push form of Sec. 4.2: unknowns are taken in level order; unknown i
// waits until its dependency counter count(i) reaches zero, finishes
// x(i) := x(i) / d(i), and then, for every unknown r that depends on it
// (column i of the matrix, read as row i of the CSR of its transpose),
// subtracts a(r, i) x(i) from x(r) and decrements count(r).  Partial sums
// are thus applied as soon as each dependency is known (the "more
// aggressive" schedule of Fig. 2), at the price of atomic updates: the order
// in which contributions reach x(r) is not fixed, so results agree with the
// row-wise solve to rounding but are not bitwise reproducible.
//
// GB300 form (the paper's CUDA kernel is prior art, not the blueprint):
//  * tickets from an atomic counter instead of the warp index (no residency
//    assumption), rows in jlev order as in the paper;
//  * a sub-warp of W lanes per unknown (32/W unknowns per warp), all lanes
//    of the warp in converged polling rounds (no lane-0 spin relying on
//    lockstep);
//  * the contribution is a relaxed FP64 atomic add and the counter
//    decrement a release atomic, so no separate fence is issued; the waiting
//    unknown reads its counter with an acquire load and then its accumulated
//    x(i);
//  * every wait is bounded: past the limit the unknown records
//    SPTRSV_ERR_TIMEOUT, finishes with NaN and still pushes, so every later
//    unknown completes.
#include "internal.h"

namespace sptrsv {

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_dec(int* p) {
    asm volatile("red.release.gpu.global.add.s32 [%0], -1;" ::"l"(p) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
    asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ void red_add(float* p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// count[r] = off-diagonal entries of row r of the system matrix (its
// dependencies); the row structure is ptr/idx.
__global__ void column_counts_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                int* count) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        int c = 0;
        for (int q = ptr[r]; q < ptr[r + 1]; ++q) c += idx[q] != (int)r;
        count[r] = c;
    }
}

cudaError_t launch_column_counts(int n, const int* ptr, const int* idx, int* count,
                                 cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 65535) g = 65535;
    column_counts_k<<<(int)g, 256, 0, s>>>(n, ptr, idx, count);
    return cudaGetLastError();
}

// x = b (the accumulator starts as the right-hand side), count = count0,
// ticket = 0.
template <typename T>
__global__ void prep_column_k(int n, T* x, long long ldx, const T* b, long long ldb,
                              const int* __restrict__ count0, int* count, int* ticket) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        if (x != b) x[r * ldx] = b[r * ldb];
        count[r] = count0[r];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;
}

// c.ptr/c.idx/c.vmap: CSR of the transpose of the system matrix, i.e. the
// column structure: row i lists the unknowns r that depend on i (and i
// itself, the diagonal, first for a lower system's transpose, last for an
// upper one's: c.diag_first).
template <typename T, int W, bool CMAP>
__global__ void __launch_bounds__(1024) column_solve_k1(SolveParams p, ColumnParams c) {
    constexpr int R = 32 / W;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const T* __restrict__ vals = (const T*)p.vals;
    T* x = (T*)p.x;
    int* count = c.count;
    int t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while ((long long)t * R < p.n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(p.ticket, 1);
        const long long k = (long long)t * R + grp;
        const bool has_row = k < p.n;
        int i = 0, cb = 0, ce = 0;
        T dinv = T(1);
        if (has_row) {
            i = p.jlev[k];
            cb = c.ptr[i];
            ce = c.ptr[i + 1];
            if (sl == 0 && !p.unit) {  // 1/d(i) while the dependencies are pending
                const int qd = c.diag_first ? cb : ce - 1;
                dinv = T(1) / vals[CMAP ? c.vmap[qd] : qd];
            }
        }
        bool done = !has_row;
        long long waits = 0;
        unsigned ns = 32;
        while (true) {
            bool ready = false, late = false;
            if (!done && i == p.withhold) {
                done = true;  // test hook: this unknown never pushes
            } else if (!done && sl == 0) {
                ready = ld_acquire(count + i) == 0;
                if (!ready && waits + 1 >= p.spin.limit) {
                    report(p.status, i, kCodeTimeout);
                    ready = late = true;
                }
            }
            ready = __shfl_sync(FULL, ready, grp * W);
            if (__any_sync(FULL, ready)) {
                T xi = T(0);
                if (ready && sl == 0) {
                    xi = late ? Marker<T>::canonical_nan() : ld_relaxed(x + (long long)i * p.ldx);
                    if (!p.unit) xi *= dinv;
                }
                xi = __shfl_sync(FULL, xi, grp * W);
                if (ready) {
                    // push a(r, i) x(i) to every dependent r; the release on
                    // the counter orders the add before it
                    for (int q = cb + sl; q < ce; q += W) {
                        const int r = c.idx[q];
                        if (r == i) continue;
                        red_add(x + (long long)r * p.ldx, -vals[CMAP ? c.vmap[q] : q] * xi);
                        red_release_dec(count + r);
                    }
                    if (sl == 0) x[(long long)i * p.ldx] = xi;
                    done = true;
                }
                waits = 0;
                ns = 32;
            } else if (++waits >= p.spin.hot) {
                __nanosleep(ns);
                ns = ns < p.spin.max_ns ? ns * 2 : p.spin.max_ns;
            }
            if (__all_sync(FULL, done)) break;
        }
        t = __shfl_sync(FULL, tn, 0);
    }
}

template <typename T, int W>
static cudaError_t column_w(const SolveParams& p, const ColumnParams& c, int grid, int block,
                            cudaStream_t s) {
    if (c.vmap)
        column_solve_k1<T, W, true><<<grid, block, 0, s>>>(p, c);
    else
        column_solve_k1<T, W, false><<<grid, block, 0, s>>>(p, c);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t column_t(int lanes, const SolveParams& p, const ColumnParams& c, int grid,
                            int block, cudaStream_t s) {
    switch (lanes) {
        case 1: return column_w<T, 1>(p, c, grid, block, s);
        case 2: return column_w<T, 2>(p, c, grid, block, s);
        case 4: return column_w<T, 4>(p, c, grid, block, s);
        case 8: return column_w<T, 8>(p, c, grid, block, s);
        case 16: return column_w<T, 16>(p, c, grid, block, s);
        case 32: return column_w<T, 32>(p, c, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_prep_column(bool f64, const SolveParams& p, const ColumnParams& c, int grid,
                               cudaStream_t s) {
    long long want = ((long long)p.n + 255) / 256;
    int g = (int)(want < grid ? want : grid);
    if (g < 1) g = 1;
    if (f64)
        prep_column_k<double><<<g, 256, 0, s>>>(p.n, (double*)p.x, p.ldx, (const double*)p.b,
                                                p.ldb, c.count0, c.count, p.ticket);
    else
        prep_column_k<float><<<g, 256, 0, s>>>(p.n, (float*)p.x, p.ldx, (const float*)p.b,
                                               p.ldb, c.count0, c.count, p.ticket);
    return cudaGetLastError();
}

cudaError_t launch_column_k1(bool f64, int lanes, const SolveParams& p, const ColumnParams& c,
                             int grid, int block, cudaStream_t s) {
    return f64 ? column_t<double>(lanes, p, c, grid, block, s)
               : column_t<float>(lanes, p, c, grid, block, s);
}

template <typename T, bool CMAP>
static int occ_col(int lanes, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SPTRSV_OCC(WW) \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, column_solve_k1<T, WW, CMAP>, block, 0)
    switch (lanes) {
        case 1: SPTRSV_OCC(1); break;
        case 2: SPTRSV_OCC(2); break;
        case 4: SPTRSV_OCC(4); break;
        case 8: SPTRSV_OCC(8); break;
        case 16: SPTRSV_OCC(16); break;
        case 32: SPTRSV_OCC(32); break;
    }
#undef SPTRSV_OCC
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int column_blocks_per_sm(bool f64, int lanes, bool cmap, int block) {
    if (f64) return cmap ? occ_col<double, true>(lanes, block) : occ_col<double, false>(lanes, block);
    return cmap ? occ_col<float, true>(lanes, block) : occ_col<float, false>(lanes, block);
}

}  // namespace sptrsv
