// Level-scheduled solve (Alg. 1, LEVR) for one right-hand side: one launch
// per level, the launch boundary being the global synchronisation between
// levels (Sec. 4.3).  Every row of the level is reduced by a sub-warp of W
// lanes with shuffles (the paper's LEVR uses a whole warp and a shared-memory
// tree).  The baseline form the self-scheduled solve is measured against.
#include "internal.h"

namespace sptrsv {

template <typename T, int W, bool MAP>
__global__ void __launch_bounds__(1024) level_solve_k1(SolveParams p) {
    const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / W;
    if (g >= p.cnt) return;  // whole sub-warps leave together
    const int lane = threadIdx.x & 31;
    const int sl = lane % W;
    const unsigned gmask = group_mask<W>(lane);
    const T* __restrict__ vals = (const T*)p.vals;
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    const int i = p.jlev[p.kbeg + g];
    const int beg = p.ptr[i], end = p.ptr[i + 1];
    T sum = T(0);
    for (int q = beg + sl; q < end; q += W) {
        const int c = p.idx[q];
        if (c != i) sum += vals[MAP ? p.vmap[q] : q] * x[(long long)c * p.ldx];
    }
    sum = group_sum<W>(sum, gmask);
    if (sl == 0) {
        T xi = b[(long long)i * p.ldb] - sum;
        if (!p.unit) {
            const int q = p.diag_first ? beg : end - 1;
            xi = xi / vals[MAP ? p.vmap[q] : q];
        }
        x[(long long)i * p.ldx] = xi;
    }
}

template <typename T, int W>
static cudaError_t level_w(const SolveParams& p, int block, cudaStream_t s) {
    const long long threads = (long long)p.cnt * W;
    const int grid = (int)((threads + block - 1) / block);
    if (p.vmap)
        level_solve_k1<T, W, true><<<grid, block, 0, s>>>(p);
    else
        level_solve_k1<T, W, false><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t level_t(int lanes, const SolveParams& p, int block, cudaStream_t s) {
    switch (lanes) {
        case 1: return level_w<T, 1>(p, block, s);
        case 2: return level_w<T, 2>(p, block, s);
        case 4: return level_w<T, 4>(p, block, s);
        case 8: return level_w<T, 8>(p, block, s);
        case 16: return level_w<T, 16>(p, block, s);
        case 32: return level_w<T, 32>(p, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_level_k1(bool f64, int lanes, const SolveParams& p, int block, cudaStream_t s) {
    return f64 ? level_t<double>(lanes, p, block, s) : level_t<float>(lanes, p, block, s);
}

}  // namespace sptrsv
