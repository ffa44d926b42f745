// Blocked self-scheduled solve, one right-hand side: on the plan's
// level-ordered copy (SPTRSV_ALGO_SELF_BLOCKED) or, one part per tile, on its
// part-ordered copy (SPTRSV_ALGO_SELF_PARTITIONED, solve_parts.cu).
//
// When levels are narrow (tens to hundreds of rows), a solve is a long chain
// of small steps and every step of Alg. 3 pays an L2 handshake (~0.6-0.8 us
// on GB300).  In level order consecutive levels are consecutive positions,
// so a tile of T consecutive positions holds many whole levels, and most
// dependencies of a row point into the same tile.  A thread block takes a
// tile (tickets, as rows are taken in Alg. 3) and:
//  * serves a dependency inside the tile from a shared-memory copy of the
//    tile's results (Sec. 4.3 remark 2: consecutive warps on consecutive
//    unknowns make shared-memory partial results possible once the matrix is
//    preordered by level); dependencies on earlier tiles are polled in the
//    position-ordered publication buffer in global memory, as in Alg. 3;
//  * hands its warps groups of 32/W consecutive positions from a
//    shared-memory counter, so a slow group holds back only the rows that
//    really depend on it;
//  * prefetches the tile's rows into L2 in a window two rounds of groups
//    ahead of the groups being taken, so their loads are L2 hits when the
//    groups start.
// A block starts its next tile only when every group of the current one is
// done (one block barrier per tile); that tile is not yet on the critical
// path when this happens.  Deadlock freedom: a group waits only on earlier
// positions, i.e. on groups of this tile taken earlier by running warps of
// this block or on earlier tiles held by running blocks.  Every wait is
// bounded.  Each row is reduced in the same order as in the other
// self-scheduled forms, so results are bitwise equal for the same sub-warp
// width.  With one lane per row a row is published right after its last
// fold (no lane reduction to wait for).  Optionally (CS > 1) thread-block
// clusters of CS blocks take CS consecutive tiles together and read each
// other's tiles in distributed shared memory.
#include "internal.h"

namespace sptrsv {

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename T>
__device__ __forceinline__ T lds_volatile(const T* p) {
    return *(const volatile T*)p;
}
template <typename T>
__device__ __forceinline__ void sts_volatile(T* p, T v) {
    *(volatile T*)p = v;
}

// ---- thread-block clusters: distributed shared memory of the cluster's blocks
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Every thread of every block of the cluster; orders shared-memory accesses
// around it across the cluster.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;"
                 ::: "memory");
}
// Address of `local` (this block's shared memory) in block `rank`'s.
__device__ __forceinline__ unsigned cluster_addr(const void* local, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ double ld_cluster(unsigned a, double) {
    unsigned long long v;
    asm volatile("ld.relaxed.cluster.shared::cluster.b64 %0, [%1];" : "=l"(v) : "r"(a) : "memory");
    return __longlong_as_double((long long)v);
}
__device__ __forceinline__ float ld_cluster(unsigned a, float) {
    unsigned v;
    asm volatile("ld.relaxed.cluster.shared::cluster.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return __uint_as_float(v);
}
__device__ __forceinline__ int ld_cluster_int(unsigned a) {
    int v;
    asm volatile("ld.relaxed.cluster.shared::cluster.b32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
// Publication into this block's shared memory, visible to the cluster.
__device__ __forceinline__ void st_cluster(double* p, double v) {
    asm volatile("st.relaxed.cluster.shared::cta.b64 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(p)),
                 "l"((unsigned long long)__double_as_longlong(v))
                 : "memory");
}
__device__ __forceinline__ void st_cluster(float* p, float v) {
    asm volatile("st.relaxed.cluster.shared::cta.b32 [%0], %1;" ::"r"(
                     (unsigned)__cvta_generic_to_shared(p)),
                 "r"(__float_as_uint(v))
                 : "memory");
}

// CS > 1: a cluster of CS blocks takes CS consecutive tiles at once (one
// ticket), block r the r-th; a dependency on one of the earlier tiles of the
// same group is read from that block's shared memory (distributed shared
// memory, no L2 round trip), one on an earlier group from the publication
// buffer.  Three cluster barriers per group: after the ticket is taken,
// after every block has read it and reset its tile (no block reads a stale
// tile of another), and when every block is done (no block reuses, or exits
// with, shared memory another still reads).
template <typename T, int W, int CS>
__global__ void __launch_bounds__(1024) blocked_solve_k1(SolveParams p, int tile_rows) {
    extern __shared__ __align__(16) unsigned char blocked_smem[];
    T* xs = (T*)blocked_smem;
    __shared__ int s_tile;
    __shared__ int s_next;
    __shared__ long long s_pst[CS];  // first position of each tile of the cluster's group
    const unsigned crank = CS > 1 ? cluster_rank() : 0u;
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    const T* __restrict__ vals = (const T*)p.vals;  // level-ordered copy
    const T* b = (const T*)p.b;
    T* x = (T*)p.x;
    T* xp = (T*)p.xp;  // publication buffer, position order
    const int n = p.n;
    // First position of tile j (tiles of tile_rows positions, or the part
    // boundaries of p.part_ptr); n past the last tile.
    auto tile_start = [&](long long j) -> long long {
        if (p.part_ptr) return j < p.nparts ? (long long)p.part_ptr[j] : (long long)n;
        const long long q = j * tile_rows;
        return q < n ? q : (long long)n;
    };
    while (true) {
        long long p0, g0 = 0;  // this block's tile, and its group's first position
        int in_tile;
        if (CS == 1) {
            if (threadIdx.x == 0) {
                s_tile = atomicAdd(p.ticket, 1);
                s_next = 0;
            }
            __syncthreads();
            p0 = tile_start(s_tile);
            if (p0 >= n) break;
            in_tile = (int)(tile_start((long long)s_tile + 1) - p0);
        } else {
            if (crank == 0 && threadIdx.x == 0) s_tile = atomicAdd(p.ticket, 1);
            cluster_sync();
            const long long t = crank == 0 ? s_tile : ld_cluster_int(cluster_addr(&s_tile, 0));
            g0 = tile_start(t * CS);
            p0 = tile_start(t * CS + crank);
            in_tile = (int)(tile_start(t * CS + crank + 1) - p0);
            if (threadIdx.x < CS) s_pst[threadIdx.x] = tile_start(t * CS + threadIdx.x);
            if (threadIdx.x == 0) s_next = 0;
            for (int k = threadIdx.x; k < in_tile; k += blockDim.x)
                xs[k] = Marker<T>::pending_value();
            cluster_sync();
            if (g0 >= n) break;  // the same for the whole cluster
        }
        if (CS == 1)
            for (int k = threadIdx.x; k < in_tile; k += blockDim.x)
                xs[k] = Marker<T>::pending_value();
        // L2 prefetch of the tile's rows (contiguous in the copy), one 128-byte
        // line per request, in a window that stays two rounds of groups ahead
        // of the groups being taken: the first rows now, the rest as groups are
        // taken.  Prefetching the whole tile at once made concurrent tiles
        // evict each other's lines (and the published values) from L2.
        const int pf_rows = (int)(blockDim.x >> 5) * R * 2;
        if (in_tile > 0) {
            const int m = in_tile < pf_rows ? in_tile : pf_rows;
            const long long q0 = p.ptr[p0], q1 = p.ptr[p0 + m];
            for (long long q = q0 + 32ll * threadIdx.x; q < q1; q += 32ll * blockDim.x)
                prefetch_l2(p.idx + q);
            for (long long q = q0 + (128 / sizeof(T)) * threadIdx.x; q < q1;
                 q += (long long)(128 / sizeof(T)) * blockDim.x)
                prefetch_l2(vals + q);
        }
        __syncthreads();
        const int groups = (in_tile + R - 1) / R;
        while (true) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&s_next, 1);
            g = __shfl_sync(FULL, g, 0);
            if (g >= groups) break;
            {   // keep the prefetch window: the rows pf_rows positions ahead
                const int a0 = g * R + pf_rows;
                if (a0 < in_tile) {
                    const int a1 = a0 + R < in_tile ? a0 + R : in_tile;
                    const long long q0 = p.ptr[p0 + a0], q1 = p.ptr[p0 + a1];
                    for (long long q = q0 + 32ll * lane; q < q1; q += 32ll * 32)
                        prefetch_l2(p.idx + q);
                    for (long long q = q0 + (128 / sizeof(T)) * lane; q < q1;
                         q += (long long)(128 / sizeof(T)) * 32)
                        prefetch_l2(vals + q);
                }
            }
            const int off = g * R + grp;  // this lane group's position in the tile
            const long long k = p0 + off;
            const bool has_row = off < in_tile;
            int i = 0, beg = 0, end = 0;
            T dinv = T(1), sum = T(0);
            double xbase = 0.0;  // refinement: the solution the row's value is added to
            if (has_row) {
                i = p.jlev[k];
                beg = p.ptr[k];
                end = p.ptr[k + 1];
                if (sl == 0) {  // same arithmetic as the other self-scheduled forms
                    if (!p.unit) {
                        const int q = p.diag_first ? beg : end - 1;
                        dinv = p.prescaled ? vals[q] : T(1) / vals[q];  // copy may hold 1/d(i)
                    }
                    sum = b[(long long)i * p.ldb];
                    if (!p.unit) sum *= dinv;
                    xbase = accumulate_base(p, i, 0);
                }
            }
            if (W > 1 && !p.unit && !p.prescaled) dinv = __shfl_sync(FULL, dinv, grp * W);
            const int span = warp_span<W>(has_row, end - beg);
            int q0 = beg + sl;
            // position of the dependency, its offset in the tile, or (remote)
            // its address in another block's shared memory
            int c[E];
            T a[E], v[E];
            unsigned live = 0, pend = 0, local = 0, remote = 0;
            auto poll = [&](int e) -> T {
                if (local & (1u << e)) return lds_volatile(xs + c[e]);
                if (CS > 1 && (remote & (1u << e))) return ld_cluster((unsigned)c[e], T(0));
                return ld_relaxed(xp + c[e]);
            };
            auto load_chunk = [&]() {
                live = pend = local = remote = 0;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int q = q0 + e * W;
                    c[e] = -1;
                    a[e] = T(0);
                    v[e] = T(0);
                    if (q < end) {
                        const int cc = p.idx[q];
                        if (cc != (int)k) {
                            a[e] = vals[q];
                            live |= 1u << e;
                            if (cc >= p0) {
                                c[e] = (int)(cc - p0);
                                local |= 1u << e;
                            } else if (CS > 1 && cc >= g0) {
                                // the earlier tile of the group that holds cc
                                unsigned r = 0;
#pragma unroll
                                for (int j = 1; j < CS; ++j)
                                    if (j < (int)crank && s_pst[j] <= cc) r = (unsigned)j;
                                c[e] = (int)cluster_addr(xs + (int)(cc - s_pst[r]), r);
                                remote |= 1u << e;
                            } else {
                                c[e] = cc;
                            }
                        }
                    }
                }
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (!(live & (1u << e))) continue;
                    v[e] = poll(e);
                }
                if (!p.unit && !p.prescaled) {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (live & (1u << e)) a[e] *= dinv;
                }
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((live & (1u << e)) && Marker<T>::pending(v[e])) pend |= 1u << e;
            };
            // one lane per row: store the row's value (shared memory, the
            // publication buffer and x)
            auto publish_row = [&](T tot) {
                const T xi = publishable(tot);
                if (CS > 1)
                    st_cluster(xs + off, xi);
                else
                    sts_volatile(xs + off, xi);
                st_relaxed(xp + k, xi);
                if (p.xacc)
                    accumulate_with(p, i, 0, xi, xbase);
                else
                    x[(long long)i * p.ldx] = xi;
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
                    if (q0 >= end) {
                        lane_done = true;
                        // one lane per row: the row is complete, publish it at
                        // once (no lane reduction to wait for)
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
                if (__any_sync(FULL, fresh)) {
                    const T tot = group_sum_span<W>(sum, FULL, span);
                    if (fresh && sl == 0 && i != p.withhold) publish_row(tot);
                }
                published = published || fresh;
                if (__all_sync(FULL, published)) break;
                if (__any_sync(FULL, !lane_done && pend == 0)) continue;  // fold first
                if (__any_sync(FULL, pend != 0)) {
                    // Tight wait: re-poll the pending entries (shared memory or
                    // the publication buffer) until something arrives.
                    const unsigned before = pend;
                    do {
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            if (!(pend & (1u << e))) continue;
                            v[e] = poll(e);
                        }
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if ((pend & (1u << e)) && !Marker<T>::pending(v[e]))
                                pend &= ~(1u << e);
                        // one lane per row and this was the row's last chunk:
                        // fold and publish now, before the warp leaves the wait
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
                            // rows of one lane publish inside the loop: leave it
                            // only when every lane is done or one needs its next
                            // chunk (one warp reduction per round)
                            const unsigned w = __reduce_or_sync(
                                FULL, lane_done ? 0u : (pend != 0 ? 1u : 2u));
                            if ((w & 2u) || !(w & 1u)) break;
                        } else if (__any_sync(FULL, pend != before)) {
                            break;
                        }
                        if (waits >= p.spin.hot &&
                            __any_sync(FULL, (pend & ~local & ~remote) != 0)) {
                            __nanosleep(ns);  // back off only while an L2 dependency is pending
                            ns = ns < p.spin.max_ns ? ns * 2 : p.spin.max_ns;
                        }
                    } while (true);
                } else {
                    waits = 0;
                    ns = 32;
                }
            }
        }
        if (CS == 1)
            __syncthreads();  // every group of the tile is done before xs is reused
        else
            cluster_sync();  // ... and no other block of the cluster still reads it
    }
}

// Lets blocked_solve_k1<T, W, CS> take the device's opt-in shared memory
// (tiles beyond 48 KB; once per device).
template <typename T, int W, int CS>
static cudaError_t blocked_attrs() {
    static unsigned long long done = 0;  // one bit per device
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done & bit) return cudaSuccess;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(blocked_solve_k1<T, W, CS>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 128);
    if (e == cudaSuccess) done |= bit;
    return e;
}

template <int CS>
static cudaLaunchConfig_t blocked_config(int grid, int block, size_t smem, cudaStream_t s,
                                         cudaLaunchAttribute* attr) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)block, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <typename T, int W, int CS>
static cudaError_t blocked_w(const SolveParams& p, int tile_rows, int grid, int block,
                             cudaStream_t s) {
    const size_t smem = sizeof(T) * (size_t)tile_rows;  // checked by the caller
    if (smem > 48 * 1024 - 256 || CS > 1) {
        cudaError_t e = blocked_attrs<T, W, CS>();
        if (e != cudaSuccess) return e;
    }
    if (CS == 1) {
        blocked_solve_k1<T, W, 1><<<grid, block, smem, s>>>(p, tile_rows);
        return cudaGetLastError();
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = blocked_config<CS>(grid, block, smem, s, attr);  // grid % CS == 0
    return cudaLaunchKernelEx(&cfg, blocked_solve_k1<T, W, CS>, p, tile_rows);
}

template <typename T, int W>
static cudaError_t blocked_c(int cluster, const SolveParams& p, int tile_rows, int grid,
                             int block, cudaStream_t s) {
    switch (cluster) {
        case 1: return blocked_w<T, W, 1>(p, tile_rows, grid, block, s);
        case 2: return blocked_w<T, W, 2>(p, tile_rows, grid, block, s);
        case 4: return blocked_w<T, W, 4>(p, tile_rows, grid, block, s);
        case 8: return blocked_w<T, W, 8>(p, tile_rows, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t blocked_t(int lanes, int cluster, const SolveParams& p, int tile_rows,
                             int grid, int block, cudaStream_t s) {
    switch (lanes) {
        case 1: return blocked_c<T, 1>(cluster, p, tile_rows, grid, block, s);
        case 2: return blocked_c<T, 2>(cluster, p, tile_rows, grid, block, s);
        case 4: return blocked_c<T, 4>(cluster, p, tile_rows, grid, block, s);
        case 8: return blocked_c<T, 8>(cluster, p, tile_rows, grid, block, s);
        case 16: return blocked_c<T, 16>(cluster, p, tile_rows, grid, block, s);
        case 32: return blocked_c<T, 32>(cluster, p, tile_rows, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_blocked_k1(bool f64, int lanes, const SolveParams& p, int tile_rows, int grid,
                              int block, cudaStream_t s, int cluster) {
    return f64 ? blocked_t<double>(lanes, cluster, p, tile_rows, grid, block, s)
               : blocked_t<float>(lanes, cluster, p, tile_rows, grid, block, s);
}

// Resident blocks of one launch: per SM times SMs without clusters, whole
// clusters times the cluster size with them.
template <typename T, int W, int CS>
static int occ_blocked_w(int block, size_t smem, int num_sms) {
    if ((smem > 48 * 1024 - 256 || CS > 1) && blocked_attrs<T, W, CS>() != cudaSuccess) return 0;
    if (CS == 1) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, blocked_solve_k1<T, W, 1>, block,
                                                          smem) != cudaSuccess)
            return 0;
        return nb * num_sms;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = blocked_config<CS>(CS, block, smem, nullptr, attr);
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, blocked_solve_k1<T, W, CS>, &cfg) != cudaSuccess)
        return 0;
    return nc * CS;
}

template <typename T, int W>
static int occ_blocked_c(int cluster, int block, size_t smem, int num_sms) {
    switch (cluster) {
        case 1: return occ_blocked_w<T, W, 1>(block, smem, num_sms);
        case 2: return occ_blocked_w<T, W, 2>(block, smem, num_sms);
        case 4: return occ_blocked_w<T, W, 4>(block, smem, num_sms);
        case 8: return occ_blocked_w<T, W, 8>(block, smem, num_sms);
        default: return 0;
    }
}

template <typename T>
static int occ_blocked(int lanes, int cluster, int block, size_t smem, int num_sms) {
    switch (lanes) {
        case 1: return occ_blocked_c<T, 1>(cluster, block, smem, num_sms);
        case 2: return occ_blocked_c<T, 2>(cluster, block, smem, num_sms);
        case 4: return occ_blocked_c<T, 4>(cluster, block, smem, num_sms);
        case 8: return occ_blocked_c<T, 8>(cluster, block, smem, num_sms);
        case 16: return occ_blocked_c<T, 16>(cluster, block, smem, num_sms);
        case 32: return occ_blocked_c<T, 32>(cluster, block, smem, num_sms);
        default: return 0;
    }
}

int blocked_resident_blocks(bool f64, int lanes, int cluster, int block, int tile_rows,
                            int num_sms) {
    const size_t smem = (f64 ? 8 : 4) * (size_t)tile_rows;
    return f64 ? occ_blocked<double>(lanes, cluster, block, smem, num_sms)
               : occ_blocked<float>(lanes, cluster, block, smem, num_sms);
}

}  // namespace sptrsv
