// Chained self-scheduled solve (SPTRSV_ALGO_SELF_CHAINS), one right-hand side.
//
// Every dependency the level-ordered solve (Alg. 3) crosses costs an L2
// handshake, ~1.5 us on GB300.  Here a ticket is a segment of R = 32/W
// consecutive rows in substitution order (natural order, reversed for
// upper).  Rows of a segment are often chained (a grid line, a band), and a
// dependency inside the segment is handed from lane to lane by shuffle as
// soon as the source row is reduced, without touching memory.  Out-of-segment
// dependencies are polled in x exactly as in the level-ordered kernel.
//
// Tickets are taken in `torder`: segments sorted by their level in the
// segment graph (1 + max level of the segments they depend on), which keeps
// the warps near the dependency frontier as level order does for rows.
// Deadlock freedom: every out-of-segment dependency lies in a segment of
// strictly lower segment level, i.e. in an earlier ticket held by a running
// warp; in-segment dependencies point to earlier lanes of the same warp,
// which publish inside the same converged round loop.
#include "internal.h"

namespace sptrsv {

template <typename T, int W, bool MAP>
__global__ void __launch_bounds__(1024) chain_solve_k1(SolveParams p,
                                                       const int* __restrict__ torder) {
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    const bool rev = p.diag_first;  // upper pattern: substitution order is n-1 .. 0
    const bool rvs = rev;  // farthest dependency first: an upper row from its last entry back
    const T* __restrict__ vals = (const T*)p.vals;
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    const int n = p.n;
    const long long nseg = ((long long)n + R - 1) / R;
    int t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while (t < nseg) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(p.ticket, 1);
        const long long p0 = (long long)torder[t] * R;  // first position of the segment
        const long long pos = p0 + grp;
        const bool has_row = pos < n;
        int i = 0, beg = 0, end = 0;
        T dinv = T(1), sum = T(0);
        if (has_row) {
            i = rev ? (int)(n - 1 - pos) : (int)pos;
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
        int c[E];  // column, or for an in-segment dependency the source lane group
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
                        const long long cp = rev ? (long long)(n - 1 - cc) : (long long)cc;
                        if (cp >= p0) {
                            c[e] = (int)(cp - p0);
                            local |= 1u << e;
                        } else {
                            c[e] = cc;
                        }
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((live & ~local) & (1u << e)) v[e] = ld_relaxed(x + (long long)c[e] * p.ldx);
            if (!p.unit) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (live & (1u << e)) a[e] *= dinv;
            }
            pend = live & local;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (((live & ~local) & (1u << e)) && Marker<T>::pending(v[e])) pend |= 1u << e;
        };
        bool lane_done = q0 >= end;
        if (!lane_done) load_chunk();
        bool published = !has_row;
        T pubv = T(0);  // this group's value once reduced (held by all its lanes)
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
            const bool fresh = !published && (done & gmask) == gmask;
            if (__any_sync(FULL, fresh)) {
                const T tot = group_sum<W>(sum, FULL);
                if (fresh) {
                    pubv = publishable(tot);
                    if (sl == 0 && i != p.withhold) st_relaxed(x + (long long)i * p.ldx, pubv);
                }
            }
            published = published || fresh;
            if (__all_sync(FULL, published)) break;
            // in-segment dependencies: take the source group's value by shuffle
            // (a withheld row, the test hook, is never forwarded either)
            const unsigned pub_lanes = __ballot_sync(FULL, published && i != p.withhold);
            if (__any_sync(FULL, (pend & local) != 0)) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const bool want = (pend & local & (1u << e)) != 0;
                    const int src = (want ? c[e] : grp) * W;
                    const T got = __shfl_sync(FULL, pubv, src);
                    if (want && ((pub_lanes >> src) & 1u)) {
                        v[e] = got;
                        pend &= ~(1u << e);
                    }
                }
            }
            if (__any_sync(FULL, !lane_done && pend == 0)) continue;  // fold first
            // Tight wait on out-of-segment dependencies (one vote per poll).
            if (__any_sync(FULL, (pend & ~local) != 0)) {
                const unsigned before = pend;
                do {
                    const unsigned far = pend & ~local;
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (far & (1u << e)) v[e] = ld_relaxed(x + (long long)c[e] * p.ldx);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if ((far & (1u << e)) && !Marker<T>::pending(v[e])) pend &= ~(1u << e);
                    if (++waits >= p.spin.limit) {
                        const unsigned still = pend & ~local;
                        if (still) {
                            report(p.status, i, kCodeTimeout);
#pragma unroll
                            for (int e = 0; e < E; ++e)
                                if (still & (1u << e)) v[e] = Marker<T>::canonical_nan();
                            pend &= local;
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
            } else if (++waits >= p.spin.limit) {
                // Only in-segment dependencies are missing.  The lowest
                // unpublished group always folds or waits on x, so this is
                // reached only when a source row is withheld: that group gives
                // up as a timed-out wait does, the later ones then go on.
                const unsigned unpub = ~__ballot_sync(FULL, published);
                if (grp == (__ffs(unpub) - 1) / W && pend) {
                    report(p.status, i, kCodeTimeout);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (pend & (1u << e)) v[e] = Marker<T>::canonical_nan();
                    pend = 0;
                }
                waits = 0;
            }
        }
        t = __shfl_sync(FULL, tn, 0);
    }
}

template <typename T, int W>
static cudaError_t chain_w(const SolveParams& p, const int* torder, int grid, int block,
                           cudaStream_t s) {
    if (p.vmap)
        chain_solve_k1<T, W, true><<<grid, block, 0, s>>>(p, torder);
    else
        chain_solve_k1<T, W, false><<<grid, block, 0, s>>>(p, torder);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t chain_t(int lanes, const SolveParams& p, const int* torder, int grid,
                           int block, cudaStream_t s) {
    switch (lanes) {
        case 1: return chain_w<T, 1>(p, torder, grid, block, s);
        case 2: return chain_w<T, 2>(p, torder, grid, block, s);
        case 4: return chain_w<T, 4>(p, torder, grid, block, s);
        case 8: return chain_w<T, 8>(p, torder, grid, block, s);
        case 16: return chain_w<T, 16>(p, torder, grid, block, s);
        case 32: return chain_w<T, 32>(p, torder, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_chain_k1(bool f64, int lanes, const SolveParams& p, const int* torder,
                            int grid, int block, cudaStream_t s) {
    return f64 ? chain_t<double>(lanes, p, torder, grid, block, s)
               : chain_t<float>(lanes, p, torder, grid, block, s);
}

template <typename T, bool MAP>
static int occ_chain(int lanes, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define SPTRSV_OCC(WW) \
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, chain_solve_k1<T, WW, MAP>, block, 0)
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

int chain_blocks_per_sm(bool f64, int lanes, bool map, int block) {
    if (f64) return map ? occ_chain<double, true>(lanes, block) : occ_chain<double, false>(lanes, block);
    return map ? occ_chain<float, true>(lanes, block) : occ_chain<float, false>(lanes, block);
}

}  // namespace sptrsv
