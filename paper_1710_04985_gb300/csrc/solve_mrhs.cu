// Multi-right-hand-side solves, self-scheduled (Alg. 3) or level-scheduled
// (Alg. 1).  A sub-warp of W lanes owns one row; lane l handles the
// right-hand-side columns l, l + W, ...  Each stored entry is read once per
// column tile and applied to all of them, so the matrix traffic is shared by
// the k solves (the multiple-right-hand-side case of Sec. 1).  No reduction
// is needed: each lane accumulates its own column in fold order (farthest
// dependency first: an upper row from its last entry back) and
// publishes it by itself, so in the self-scheduled form every (row, column)
// value is its own ready flag and lanes never wait for each other.
#include "internal.h"

namespace sptrsv {

// Level-scheduled row: all dependencies are final (earlier launches).
template <typename T, int W, bool MAP>
__device__ __forceinline__ void mrhs_row_level(const SolveParams& p, int i, int sl) {
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
        if (c >= p.nrhs) break;
        T acc = T(0);
        for (int q = beg; q < end; ++q) {
            const int j = p.idx[q];
            if (j == i) continue;
            acc += vals[MAP ? p.vmap[q] : q] * x[(long long)j * p.ldx + c];
        }
        T xi = b[(long long)i * p.ldb + c] - acc;
        if (!p.unit) xi = xi / di;
        x[(long long)i * p.ldx + c] = xi;
    }
}

// PERM: the pattern is the plan's level-ordered copy (position k = row
// jlev[k], columns renumbered to positions, values pre-scaled for a non-unit
// matrix); columns publish to the position-ordered buffer p.xp ([n][nrhs])
// that waiting lanes poll, so a level's unknowns are one contiguous run, and
// are stored to x (or added to p.xacc) for the caller.
template <typename T, int W, bool MAP, bool SELF, bool PERM = false>
__global__ void __launch_bounds__(1024) solve_mrhs_k(SolveParams p) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int E = kChunk;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    if (!SELF) {
        const long long g = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / W;
        if (g < p.cnt) mrhs_row_level<T, W, MAP>(p, p.jlev[p.kbeg + g], sl);
        return;
    }
    constexpr int R = 32 / W;
    const T* __restrict__ vals = (const T*)p.vals;
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    T* xpub = PERM ? (T*)p.xp : x;  // the array columns publish to and wait on
    const long long ldp = PERM ? p.nrhs : p.ldx;
    // farthest dependency first: an upper row from its last entry back (the
    // level-ordered copy already stores it that way round)
    const bool rvs = !PERM && p.diag_first;
    int t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while ((long long)t * R < p.n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(p.ticket, 1);
        const long long k = (long long)t * R + grp;
        int i = 0, beg = 0, end = 0;
        T dinv = T(1);
        int col = sl;
        bool lane_done = k >= p.n || col >= p.nrhs;
        // the row's identity in the pattern: its own column index
        const int self_col = PERM ? (int)k : 0;
        const long long pub = PERM ? k : 0;  // publication row in xpub
        if (k < p.n) {
            i = p.jlev[k];
            beg = p.ptr[PERM ? k : i];
            end = p.ptr[(PERM ? k : i) + 1];
            if (!p.unit) {  // computed while the dependencies are pending
                const int q = p.diag_first ? beg : end - 1;
                const T d = vals[MAP ? p.vmap[q] : q];
                dinv = p.prescaled ? d : T(1) / d;  // a pre-scaled copy holds 1/d(i)
            }
        }
        const long long prow = PERM ? pub : (long long)i;
        // per-lane state: column `col`, next entry q0, chunk of E entries; the
        // row is scaled by 1/d(i) so the column's value is the fold itself.
        int q0 = beg;
        int c[E];
        T a[E], v[E];
        unsigned live = 0, pend = 0;
        T acc = T(0);
        auto start_column = [&]() {
            acc = b[(long long)i * p.ldb + col];
            if (!p.unit) acc *= dinv;
        };
        auto load_chunk = [&]() {
            live = pend = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int q = q0 + e;
                c[e] = -1;
                a[e] = T(0);
                v[e] = T(0);
                if (q < end) {
                    const int pq = rvs ? beg + end - 1 - q : q;  // fold order -> storage
                    const int cc = p.idx[pq];
                    if (cc != (PERM ? self_col : i)) {
                        c[e] = cc;
                        a[e] = vals[MAP ? p.vmap[pq] : pq];
                        live |= 1u << e;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (live & (1u << e)) v[e] = ld_relaxed(xpub + (long long)c[e] * ldp + col);
            if (!p.unit && !p.prescaled) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (live & (1u << e)) a[e] *= dinv;
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((live & (1u << e)) && Marker<T>::pending(v[e])) pend |= 1u << e;
        };
        if (!lane_done) {
            start_column();
            load_chunk();
        }
        long long waits = 0;
        unsigned ns = 32;
        while (true) {
            if (!lane_done && pend == 0) {
                acc = fold_chunk(acc, a, v, live);
                q0 += E;
                if (q0 >= end) {  // column done: publish it, move to the next tile
                    if (i != p.withhold) {
                        const T val = publishable(acc);
                        st_relaxed(xpub + prow * ldp + col, val);
                        if (p.xacc)
                            accumulate_published(p, i, col, val);
                        else if (PERM)
                            x[(long long)i * p.ldx + col] = val;
                    }
                    col += W;
                    q0 = beg;
                    if (col >= p.nrhs) {
                        lane_done = true;
                    } else {
                        start_column();
                        load_chunk();
                    }
                } else {
                    load_chunk();
                }
            }
            if (__all_sync(FULL, lane_done)) break;
            if (__any_sync(FULL, !lane_done && pend == 0)) continue;  // fold first
            if (__any_sync(FULL, pend != 0)) {
                const unsigned before = pend;
                do {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (pend & (1u << e)) v[e] = ld_relaxed(xpub + (long long)c[e] * ldp + col);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if ((pend & (1u << e)) && !Marker<T>::pending(v[e])) pend &= ~(1u << e);
                    if (++waits >= p.spin.limit) {
                        if (pend) {
                            report(p.status, i, kCodeTimeout);
#pragma unroll
                            for (int e = 0; e < E; ++e)
                                if (pend & (1u << e)) v[e] = Marker<T>::canonical_nan();
                            pend = 0;
                        }
                        waits = 0;
                        break;
                    }
                    if (__any_sync(FULL, pend != before)) break;
                    if (waits >= p.spin.hot) {
                        __nanosleep(ns);
                        ns = ns < p.spin.max_ns ? ns * 2 : p.spin.max_ns;
                    }
                } while (true);
            } else {
                waits = 0;
                ns = 32;
            }
        }
        t = __shfl_sync(FULL, tn, 0);
    }
}

template <typename T, int W, bool SELF>
static cudaError_t mrhs_w(const SolveParams& p, int grid, int block, cudaStream_t s) {
    if (!SELF) {
        const long long threads = (long long)p.cnt * W;
        grid = (int)((threads + block - 1) / block);
    }
    if (SELF && p.xp)  // level-ordered copy: values gathered, no map
        solve_mrhs_k<T, W, false, true, true><<<grid, block, 0, s>>>(p);
    else if (p.vmap)
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
