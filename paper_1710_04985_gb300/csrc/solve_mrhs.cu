// Multi-right-hand-side solves, self-scheduled (Alg. 3) or level-scheduled
// (Alg. 1).  A sub-warp of W lanes owns one row; lane l handles the
// right-hand-side columns l, l + W, ...  Each stored entry is read once per
// column tile and applied to all of them, so the matrix traffic is shared by
// the k solves (the multiple-right-hand-side case of Sec. 1).  No reduction
// is needed: each lane accumulates its own columns in entry order.
#include "internal.h"

namespace sptrsv {

template <typename T, int W, bool MAP, bool SELF>
__device__ __forceinline__ void mrhs_row(const SolveParams& p, int i, int sl) {
    const T* __restrict__ vals = (const T*)p.vals;
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    const int beg = p.ptr[i], end = p.ptr[i + 1];
    T di = T(1);
    if (!p.unit) {
        const int q = p.diag_first ? beg : end - 1;
        di = vals[MAP ? p.vmap[q] : q];
    }
    for (int c0 = 0; c0 < p.nrhs; c0 += W) {
        const int c = c0 + sl;
        const bool on = c < p.nrhs;
        T acc = T(0);
        for (int q = beg; q < end; ++q) {
            const int j = p.idx[q];
            if (j == i) continue;
            const T a = vals[MAP ? p.vmap[q] : q];
            if (on) {
                const T* src = x + (long long)j * p.ldx + c;
                const T xv = SELF ? wait_value(src, p.spin, p.status, i) : *src;
                acc += a * xv;
            }
        }
        if (on) {
            T xi = b[(long long)i * p.ldb + c] - acc;
            if (!p.unit) xi = xi / di;
            T* dst = x + (long long)i * p.ldx + c;
            if (SELF) {
                if (i != p.withhold) st_relaxed(dst, publishable(xi));
            } else {
                *dst = xi;
            }
        }
    }
}

template <typename T, int W, bool MAP, bool SELF>
__global__ void __launch_bounds__(1024) solve_mrhs_k(SolveParams p) {
    const int lane = threadIdx.x & 31;
    const int sub = lane / W;
    const int sl = lane - sub * W;
    if (!SELF) {
        const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / W;
        if (g < p.cnt) mrhs_row<T, W, MAP, false>(p, p.jlev[p.kbeg + g], sl);
        return;
    }
    constexpr int R = 32 / W;
    int t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    while ((long long)t * R < p.n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(p.ticket, 1);
        const long long k = (long long)t * R + sub;
        if (k < p.n) mrhs_row<T, W, MAP, true>(p, p.jlev[k], sl);
        t = __shfl_sync(0xffffffffu, tn, 0);
    }
}

template <typename T, int W, bool SELF>
static cudaError_t mrhs_w(const SolveParams& p, int grid, int block, cudaStream_t s) {
    if (!SELF) {
        const long long threads = (long long)p.cnt * W;
        grid = (int)((threads + block - 1) / block);
    }
    if (p.vmap)
        solve_mrhs_k<T, W, true, SELF><<<grid, block, 0, s>>>(p);
    else
        solve_mrhs_k<T, W, false, SELF><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T, bool SELF>
static cudaError_t mrhs_t(int lanes, const SolveParams& p, int grid, int block, cudaStream_t s) {
    switch (lanes) {
        case 4: return mrhs_w<T, 4, SELF>(p, grid, block, s);
        case 8: return mrhs_w<T, 8, SELF>(p, grid, block, s);
        case 16: return mrhs_w<T, 16, SELF>(p, grid, block, s);
        case 32: return mrhs_w<T, 32, SELF>(p, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mrhs(bool f64, int lanes, bool self, const SolveParams& p, int grid, int block,
                        cudaStream_t s) {
    if (f64) return self ? mrhs_t<double, true>(lanes, p, grid, block, s)
                         : mrhs_t<double, false>(lanes, p, grid, block, s);
    return self ? mrhs_t<float, true>(lanes, p, grid, block, s)
                : mrhs_t<float, false>(lanes, p, grid, block, s);
}

template <typename T, bool MAP>
static int occ_mrhs(int lanes, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (lanes) {
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_mrhs_k<T, 4, MAP, true>, block, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_mrhs_k<T, 8, MAP, true>, block, 0); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_mrhs_k<T, 16, MAP, true>, block, 0); break;
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, solve_mrhs_k<T, 32, MAP, true>, block, 0); break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

int self_k1_blocks_per_sm(bool f64, int lanes, bool map, int block);

int self_blocks_per_sm(bool f64, int lanes, bool mrhs, bool map, int block) {
    if (!mrhs) return self_k1_blocks_per_sm(f64, lanes, map, block);
    if (f64) return map ? occ_mrhs<double, true>(lanes, block) : occ_mrhs<double, false>(lanes, block);
    return map ? occ_mrhs<float, true>(lanes, block) : occ_mrhs<float, false>(lanes, block);
}

}  // namespace sptrsv
