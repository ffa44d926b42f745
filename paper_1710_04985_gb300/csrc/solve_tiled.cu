// Tiled self-scheduled solve (SPTRSV_ALGO_SELF_TILED), one right-hand side.
//
// Tiles are runs of consecutive positions either of the substitution order
// (natural row order, reversed for upper) or of the level order jlev.  The
// first suits banded and chain-like matrices; the second suits deep level
// structures with few rows per level, where one tile spans many consecutive
// levels and the critical path stays inside a tile.  Both orders are
// topological, which is all the scheduling argument below needs.
//
// The self-scheduled solve of Alg. 3 pays one L2 round trip (publish, then
// the dependent's poll) for every dependency level it crosses.  On GB300 that
// is ~1.3-1.7 us per level, so matrices with many levels are bound by it.
// Sec. 4.3 (remark 2) notes that keeping partial results in shared memory
// needs consecutive warps to work on related unknowns.  This kernel gives a
// thread block a tile of consecutive rows in substitution order (tiles are
// handed out by a ticket counter, as rows are in the level-ordered solve):
//  * a dependency inside the tile is read from the tile's shared-memory copy
//    of x (tens of cycles instead of an L2 round trip);
//  * a dependency on an earlier tile is polled in global memory exactly as in
//    the level-ordered solve (x is pre-filled with the "not yet solved"
//    marker and a published value is its own flag).
// Inside the tile, warps take groups of 32/W consecutive rows round-robin and
// run the same converged round loop as the level-ordered kernel, so rows of
// one group may depend on each other.  Deadlock freedom: every dependency
// points to an earlier position, i.e. to an earlier group of this tile (held
// by a running warp of this block, each warp taking its groups in order) or
// to an earlier tile (held by a running block).  Every wait is bounded.
#include "internal.h"

namespace sptrsv {

template <typename T>
__device__ __forceinline__ T ld_shared_volatile(const T* p) {
    return *(const volatile T*)p;
}
template <typename T>
__device__ __forceinline__ void st_shared_volatile(T* p, T v) {
    *(volatile T*)p = v;
}

template <typename T, int W, bool MAP>
__global__ void __launch_bounds__(1024) tiled_solve_k1(SolveParams p, int tile_rows) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    T* xs = (T*)tile_smem;
    __shared__ int s_tile;
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    const bool rev = p.diag_first;  // upper pattern: substitution order is n-1 .. 0
    const bool rvs = rev;  // farthest dependency first: an upper row from its last entry back
    const T* __restrict__ vals = (const T*)p.vals;
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    const int n = p.n;
    while (true) {
        if (threadIdx.x == 0) s_tile = atomicAdd(p.ticket, 1);
        __syncthreads();  // also: every warp is done with the previous tile's xs
        const long long p0 = (long long)s_tile * tile_rows;  // first position of the tile
        if (p0 >= n) break;
        const int in_tile = (int)((n - p0) < tile_rows ? (n - p0) : tile_rows);
        for (int k = threadIdx.x; k < in_tile; k += blockDim.x)
            xs[k] = Marker<T>::pending_value();
        __syncthreads();
        const int groups = (in_tile + R - 1) / R;
        for (int gi = warp; gi < groups; gi += nwarps) {
            const int off = gi * R + grp;  // offset of this lane group's row in the tile
            const bool has_row = off < in_tile;
            int i = 0, beg = 0, end = 0;
            T dinv = T(1), sum = T(0);
            if (has_row) {
                const long long pos = p0 + off;
                i = p.ipos ? p.jlev[pos] : (rev ? (int)(n - 1 - pos) : (int)pos);
                beg = p.ptr[i];
                end = p.ptr[i + 1];
                if (sl == 0) {  // same arithmetic as the level-ordered kernel
                    if (!p.unit) {
                        const int q = p.diag_first ? beg : end - 1;
                        dinv = T(1) / vals[MAP ? p.vmap[q] : q];
                    }
                    sum = b[(long long)i * p.ldb];
                    if (!p.unit) sum *= dinv;
                }
            }
            if (W > 1 && !p.unit) dinv = __shfl_sync(FULL, dinv, grp * W);
            int q0 = beg + sl;
            int c[E];  // column, or for an in-tile dependency its offset in the tile
            T a[E], v[E];
            unsigned live = 0, pend = 0, local = 0;
            auto load_chunk = [&]() {
                live = pend = local = 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int q = q0 + e * W;
                    c[e] = -1;
                    a[e] = T(0);
                    v[e] = T(0);
                    if (q < end) {
                        const int pq = rvs ? beg + end - 1 - q : q;  // fold order -> storage
                        const int cc = p.idx[pq];
                        if (cc != i) {
                            a[e] = vals[MAP ? p.vmap[pq] : pq];
                            live |= 1u << e;
                            const long long cpos =
                                p.ipos ? (long long)p.ipos[cc]
                                       : (rev ? (long long)(n - 1 - cc) : (long long)cc);
                            if (cpos >= p0) {
                                c[e] = (int)(cpos - p0);
                                local |= 1u << e;
                            } else {
                                c[e] = cc;
                            }
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (!(live & (1u << e))) continue;
                    v[e] = (local & (1u << e)) ? ld_shared_volatile(xs + c[e])
                                               : ld_relaxed(x + (long long)c[e] * p.ldx);
                }
                if (!p.unit) {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (live & (1u << e)) a[e] *= dinv;
                }
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((live & (1u << e)) && Marker<T>::pending(v[e])) pend |= 1u << e;
            };
            bool lane_done = q0 >= end;
            if (!lane_done) load_chunk();
            bool published = !has_row;
            long long waits = 0;
            unsigned ns = 32;
            while (true) {
                if (!lane_done && pend == 0) {
                    sum = fold_chunk(sum, a, v, live);
                    q0 += W * E;
                    if (q0 >= end) lane_done = true;
                    else load_chunk();
                }
                const unsigned done = __ballot_sync(FULL, lane_done);
                const bool row_ready = (done & gmask) == gmask;
                const bool fresh = row_ready && !published;
                if (__any_sync(FULL, fresh)) {
                    const T tot = group_sum<W>(sum, FULL);
                    if (fresh && sl == 0 && i != p.withhold) {
                        const T xi = publishable(tot);
                        st_shared_volatile(xs + off, xi);
                        st_relaxed(x + (long long)i * p.ldx, xi);
                    }
                }
                published = published || fresh;
                if (__all_sync(FULL, published)) break;
                if (__any_sync(FULL, pend != 0)) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (!(pend & (1u << e))) continue;
                        v[e] = (local & (1u << e)) ? ld_shared_volatile(xs + c[e])
                                                   : ld_relaxed(x + (long long)c[e] * p.ldx);
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if ((pend & (1u << e)) && !Marker<T>::pending(v[e])) pend &= ~(1u << e);
                    // `waits` advances in lockstep on all lanes: the branches are uniform.
                    if (++waits >= p.spin.limit) {
                        if (pend) {
                            report(p.status, i, kCodeTimeout);
#pragma unroll
                            for (int e = 0; e < E; ++e)
                                if (pend & (1u << e)) v[e] = Marker<T>::canonical_nan();
                            pend = 0;
                        }
                    } else if (waits >= p.spin.hot && __any_sync(FULL, (pend & ~local) != 0)) {
                        __nanosleep(ns);  // back off only while an L2 dependency is pending
                        ns = ns < p.spin.max_ns ? ns * 2 : p.spin.max_ns;
                    }
                } else {
                    waits = 0;
                    ns = 32;
                }
            }
        }
    }
}

template <typename T, int W>
static cudaError_t tiled_w(const SolveParams& p, int tile_rows, int grid, int block,
                           cudaStream_t s) {
    const size_t smem = sizeof(T) * (size_t)tile_rows;  // <= 48 KB, checked by the caller
    if (p.vmap)
        tiled_solve_k1<T, W, true><<<grid, block, smem, s>>>(p, tile_rows);
    else
        tiled_solve_k1<T, W, false><<<grid, block, smem, s>>>(p, tile_rows);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t tiled_t(int lanes, const SolveParams& p, int tile_rows, int grid, int block,
                           cudaStream_t s) {
    switch (lanes) {
        case 1: return tiled_w<T, 1>(p, tile_rows, grid, block, s);
        case 2: return tiled_w<T, 2>(p, tile_rows, grid, block, s);
        case 4: return tiled_w<T, 4>(p, tile_rows, grid, block, s);
        case 8: return tiled_w<T, 8>(p, tile_rows, grid, block, s);
        case 16: return tiled_w<T, 16>(p, tile_rows, grid, block, s);
        case 32: return tiled_w<T, 32>(p, tile_rows, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tiled_k1(bool f64, int lanes, const SolveParams& p, int tile_rows, int grid,
                            int block, cudaStream_t s) {
    return f64 ? tiled_t<double>(lanes, p, tile_rows, grid, block, s)
               : tiled_t<float>(lanes, p, tile_rows, grid, block, s);
}

template <typename T, bool MAP>
static int occ_tiled(int lanes, int block, size_t smem) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SPTRSV_OCC(W)                                                                          \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tiled_solve_k1<T, W, MAP>, block, \
                                                      smem)
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

int tiled_blocks_per_sm(bool f64, int lanes, bool map, int block, int tile_rows) {
    const size_t smem = (f64 ? 8 : 4) * (size_t)tile_rows;
    if (f64) return map ? occ_tiled<double, true>(lanes, block, smem)
                        : occ_tiled<double, false>(lanes, block, smem);
    return map ? occ_tiled<float, true>(lanes, block, smem)
               : occ_tiled<float, false>(lanes, block, smem);
}

}  // namespace sptrsv
