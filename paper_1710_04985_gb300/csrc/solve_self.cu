// Self-scheduled solve (Alg. 3, SLFR) for one right-hand side.
//
// Differences from the paper's SLFR kernel (Sec. 4.3), for sm_103a:
//  * Rows are handed out in level order (jlev), as in the paper, but by a
//    ticket counter rather than by warp index: a warp takes ticket t only
//    while running, and every row it waits on belongs to a smaller ticket,
//    already held by a running warp.  No residency assumption is needed.
//  * No dependency counters and no CSC fan-out: the output x is pre-filled
//    with a marker, and each lane waits directly on the x(j) it needs with a
//    GPU-scope relaxed load.  The published value is its own ready flag, so
//    a dependency costs one L2 round trip and no fence.
//  * A row is reduced by a sub-warp of W lanes (W chosen per matrix).  The
//    paper lets lane 0 spin and relies on warp lockstep, which sm_70 and
//    later no longer guarantee.  Here the whole warp stays converged in one
//    round loop: every lane issues the loads of all its entries of a chunk
//    at once, re-polls only the pending ones each round, and a row is reduced
//    (shuffles) and published inside the loop as soon as all its lanes are
//    done.  Rows of one ticket may therefore depend on one another (a ticket
//    can straddle two levels) without deadlock, and no sub-warp waits in a
//    divergent spin that the scheduler would serialise.  Every wait is
//    bounded.
#include "internal.h"

namespace sptrsv {

template <typename T>
__global__ void prep_self_k(int n, int nrhs, T* x, long long ldx, const T* b, long long ldb,
                            T* bcopy, int* ticket) {
    const long long total = (long long)n * nrhs;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (nrhs == 1) {
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
            if (bcopy) bcopy[e] = b[e * ldb];
            x[e * ldx] = Marker<T>::pending_value();
        }
    } else {
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
            const long long r = e / nrhs;
            const long long c = e - r * nrhs;
            if (bcopy) bcopy[e] = b[r * ldb + c];
            x[r * ldx + c] = Marker<T>::pending_value();
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *ticket = 0;
}

cudaError_t launch_prep_self(bool f64, int n, int nrhs, void* x, long long ldx, const void* b,
                             long long ldb, void* bcopy, int* ticket, int grid, cudaStream_t s) {
    long long want = ((long long)n * nrhs + 255) / 256;
    int g = (int)(want < grid ? want : grid);
    if (g < 1) g = 1;
    if (f64)
        prep_self_k<double><<<g, 256, 0, s>>>(n, nrhs, (double*)x, ldx, (const double*)b, ldb,
                                              (double*)bcopy, ticket);
    else
        prep_self_k<float><<<g, 256, 0, s>>>(n, nrhs, (float*)x, ldx, (const float*)b, ldb,
                                             (float*)bcopy, ticket);
    return cudaGetLastError();
}


// PERM: the pattern is the plan's level-ordered copy (SPTRSV_ALGO_SELF_PERMUTED):
// row position k of jlev holds the entries of row jlev[k] in fold order (an
// upper row's last entry first), with column indices renumbered to positions
// and the values copied alongside (p.ptr, p.idx, p.vals), so a warp's rows and
// the unknowns they wait on are contiguous.  Results are published in p.xp (position order,
// the array that is polled) and stored to x(jlev[k]) for the caller.  The
// arithmetic and its order are those of the unpermuted kernel, so both give
// bitwise identical results for the same sub-warp width.
template <typename T, int W, bool MAP, bool PERM>
__global__ void __launch_bounds__(1024) self_solve_k1(SolveParams p) {
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    const T* __restrict__ vals = (const T*)p.vals;
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    T* xpub = PERM ? (T*)p.xp : x;  // the array rows publish to and wait on
    const long long ldp = PERM ? 1 : p.ldx;
    // Every form folds a row's entries farthest dependency first: a lower
    // row in storage order, an upper row from its last entry back (the copies
    // already store an upper row that way round).
    const bool rvs = !PERM && p.diag_first;
    int t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while ((long long)t * R < p.n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(p.ticket, 1);  // next ticket, consumed after this one
        const long long k = (long long)t * R + grp;
        const bool has_row = k < p.n;
        int i = 0, beg = 0, end = 0;
        T dinv = T(1), sum = T(0);
        double xbase = 0.0;  // refinement: the solution the row's value is added to
        // identity of the row inside the pattern: its own column index
        const int self_col = PERM ? (int)k : 0;
        if (has_row) {
            i = p.jlev[k];
            beg = p.ptr[PERM ? k : i];
            end = p.ptr[(PERM ? k : i) + 1];
            if (sl == 0) {
                // Everything that does not depend on x happens now, while the
                // dependencies are pending (SLFR computes 1/d(i) up front too):
                // the row is scaled by 1/d(i), so x(i) = b(i)/d(i) - sum of
                // (a_ij/d(i)) x(j) and only the FMA fold and the lane reduction
                // remain once the last dependency arrives.
                if (!p.unit) {
                    const int q = p.diag_first ? beg : end - 1;
                    const T d = vals[MAP ? p.vmap[q] : q];
                    dinv = p.prescaled ? d : T(1) / d;  // a pre-scaled copy holds 1/d(i)
                }
                sum = b[(long long)i * p.ldb];
                if (!p.unit) sum *= dinv;
                xbase = accumulate_base(p, i, 0);
            }
        }
        if (W > 1 && !p.unit && !p.prescaled) dinv = __shfl_sync(FULL, dinv, grp * W);
        const int span = warp_span<W>(has_row, end - beg);
        // ---- per-lane chunk state: entries q0 + e*W, e < E
        int q0 = beg + sl;
        int c[E];
        T a[E], v[E];
        unsigned live = 0, pend = 0;  // entries that count / still unpublished
        auto load_chunk = [&]() {
            live = pend = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int q = q0 + e * W;
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
                if (live & (1u << e)) v[e] = ld_relaxed(xpub + (long long)c[e] * ldp);
            if (!p.unit && !p.prescaled) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (live & (1u << e)) a[e] *= dinv;
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((live & (1u << e)) && Marker<T>::pending(v[e])) pend |= 1u << e;
        };
        // one lane per row: store the row's value (and x, on the copy)
        auto publish_row = [&](T tot) {
            const T val = publishable(tot);
            st_relaxed(xpub + (PERM ? k : (long long)i * p.ldx), val);
            if (p.xacc)
                accumulate_with(p, i, 0, val, xbase);
            else if (PERM)
                x[(long long)i * p.ldx] = val;
        };
        bool lane_done = q0 >= end;
        if (!lane_done) load_chunk();
        bool published = !has_row;
        long long waits = 0;
        unsigned ns = 32;
        while (true) {
            if (!lane_done && pend == 0) {  // fold a complete chunk in fold order
                sum = fold_chunk(sum, a, v, live);
                q0 += W * E;
                if (q0 >= end) {
                    lane_done = true;
                    // one lane per row: the row is complete, publish it at once
                    // (no lane reduction to wait for)
                    if (W == 1 && has_row && i != p.withhold) {
                        publish_row(sum);
                        published = true;
                    }
                } else {
                    load_chunk();
                }
            }
            const unsigned done = __ballot_sync(FULL, lane_done);
            const bool fresh = !published && (done & gmask) == gmask;
            if (__any_sync(FULL, fresh)) {  // FP64 is scarce on GB300: reduce only then
                const T tot = group_sum_span<W>(sum, FULL, span);
                if (fresh && sl == 0 && i != p.withhold) publish_row(tot);
            }
            published = published || fresh;
            if (__all_sync(FULL, published)) break;
            // A lane with a complete chunk folds it first (next round); only
            // when every lane is done or waiting does the warp enter the tight
            // wait, so a row of this ticket that another row waits on is
            // never held back by the wait.
            if (__any_sync(FULL, !lane_done && pend == 0)) continue;
            // Tight wait: re-poll the pending entries until something arrives
            // anywhere in the warp (one vote per poll; uniform control flow).
            if (__any_sync(FULL, pend != 0)) {
                const unsigned before = pend;
                do {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (pend & (1u << e)) v[e] = ld_relaxed(xpub + (long long)c[e] * ldp);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if ((pend & (1u << e)) && !Marker<T>::pending(v[e])) pend &= ~(1u << e);
                    // one lane per row and this was the row's last chunk: fold
                    // and publish now, before the warp leaves the wait
                    if (W == 1 && !lane_done && pend == 0 && q0 + E >= end) {
                        sum = fold_chunk(sum, a, v, live);
                        q0 += E;
                        lane_done = true;
                        if (has_row && i != p.withhold) publish_row(sum);
                        published = true;
                    }
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
                    if (W == 1) {
                        // rows of one lane publish inside the loop: leave it only
                        // when every lane is done or one needs its next chunk
                        const unsigned w = __reduce_or_sync(
                            FULL, lane_done ? 0u : (pend != 0 ? 1u : 2u));
                        if ((w & 2u) || !(w & 1u)) break;
                    } else if (__any_sync(FULL, pend != before)) {
                        break;  // something arrived
                    }
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

template <typename T, int W>
static cudaError_t self_w(const SolveParams& p, int grid, int block, cudaStream_t s) {
    if (p.xp)  // level-ordered copy: values already gathered, no map
        self_solve_k1<T, W, false, true><<<grid, block, 0, s>>>(p);
    else if (p.vmap)
        self_solve_k1<T, W, true, false><<<grid, block, 0, s>>>(p);
    else
        self_solve_k1<T, W, false, false><<<grid, block, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t self_t(int lanes, const SolveParams& p, int grid, int block, cudaStream_t s) {
    switch (lanes) {
        case 1: return self_w<T, 1>(p, grid, block, s);
        case 2: return self_w<T, 2>(p, grid, block, s);
        case 4: return self_w<T, 4>(p, grid, block, s);
        case 8: return self_w<T, 8>(p, grid, block, s);
        case 16: return self_w<T, 16>(p, grid, block, s);
        case 32: return self_w<T, 32>(p, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_self_k1(bool f64, int lanes, const SolveParams& p, int grid, int block,
                           cudaStream_t s) {
    return f64 ? self_t<double>(lanes, p, grid, block, s) : self_t<float>(lanes, p, grid, block, s);
}

template <typename T, bool MAP>
static int occ_k1(int lanes, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (lanes) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, 1, MAP, false>, block, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, 2, MAP, false>, block, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, 4, MAP, false>, block, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, 8, MAP, false>, block, 0); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, 16, MAP, false>, block, 0); break;
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, 32, MAP, false>, block, 0); break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

template <typename T>
static int occ_perm(int lanes, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SPTRSV_OCC(WW) \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, self_solve_k1<T, WW, false, true>, block, 0)
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

int self_perm_blocks_per_sm(bool f64, int lanes, int block) {
    return f64 ? occ_perm<double>(lanes, block) : occ_perm<float>(lanes, block);
}

int self_k1_blocks_per_sm(bool f64, int lanes, bool map, int block) {
    if (f64) return map ? occ_k1<double, true>(lanes, block) : occ_k1<double, false>(lanes, block);
    return map ? occ_k1<float, true>(lanes, block) : occ_k1<float, false>(lanes, block);
}

}  // namespace sptrsv
