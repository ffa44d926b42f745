// Setup phase (Sec. 4.4): validation, level analysis (Sec. 4.1), level sets,
// and the CSR of the transpose (the CSC view of Sec. 3.2).
//
// Level analysis here is not Kahn's algorithm (Sec. 4.4.1, one launch and
// one device-to-host copy per level).  It is one persistent launch that
// sweeps the rows in substitution order: lev(i) = 1 + max lev(j) is itself a
// triangular "solve" in the (max, +) semiring, so each row waits for its
// dependencies' levels exactly as the self-scheduled solve waits for their
// values, and publishes its own level as soon as it is known.
#include "internal.h"

namespace sptrsv {

// ------------------------------------------------------------ validation
// One thread per row.  Checks (Sec. 3): rowptr monotone inside [0, nnz];
// columns in range, strictly increasing, inside the declared triangle;
// unless unit, a nonzero diagonal in its place (last entry of a lower row,
// first of an upper row).
__global__ void validate_k(int n, int nnz, const int* __restrict__ ptr,
                           const int* __restrict__ idx, const void* __restrict__ vals, int f64,
                           int upper, int unit, unsigned long long* status) {
    for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n;
         ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        const int beg = ptr[i], end = ptr[i + 1];
        if ((i == 0 && beg != 0) || (i == n - 1 && end != nnz) || beg < 0 || beg > end ||
            end > nnz) {
            report(status, i, kCodeStructure);
            continue;
        }
        int prev = -1;
        bool bad = false;
        for (int q = beg; q < end; ++q) {
            const int c = idx[q];
            if (c <= prev || c >= n || (upper ? c < i : c > i)) {
                bad = true;
                break;
            }
            prev = c;
        }
        if (bad) {
            report(status, i, kCodeStructure);
            continue;
        }
        if (!unit) {
            const int q = upper ? beg : end - 1;
            if (end == beg || idx[q] != i) {
                report(status, i, kCodeZeroPivot);
                continue;
            }
            const double v = f64 ? ((const double*)vals)[q] : (double)((const float*)vals)[q];
            if (v == 0.0) report(status, i, kCodeZeroPivot);
        }
    }
}

cudaError_t launch_validate(int n, int nnz, const int* ptr, const int* idx, const void* vals,
                            bool f64, bool upper, bool unit, unsigned long long* status,
                            int grid, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    int g = (n + 255) / 256;
    if (g > grid) g = grid;
    validate_k<<<g, 256, 0, s>>>(n, nnz, ptr, idx, vals, f64, upper, unit, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ level sweep
// Sub-warps of W lanes take groups of 32/W consecutive rows (in substitution
// order) from a ticket counter.  Every dependency of a row comes earlier in
// that order, and every earlier ticket is held by a running warp, so the
// sweep cannot deadlock whatever the residency.  lev[] starts at -1
// ("unknown"); a row publishes its level with one relaxed store.  As in the
// self-scheduled solve, the warp stays converged in one round loop.  Rows of
// one ticket are consecutive, so they often depend on each other (a chain
// along a grid line, a band): such a dependency is served by a warp shuffle
// from the lane that owns the row as soon as it is published, instead of an
// L2 round trip.
template <int W>
__global__ void level_sweep_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                              int upper, int* lev, int* ticket, int* nlev,
                              unsigned long long* status, SpinPolicy sp) {
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    int local_max = -1;
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while ((long long)t * R < n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(ticket, 1);
        // rows of this ticket: first = t*R in substitution order
        const int first = (int)((long long)t * R);
        const int rows = (n - first) < R ? (n - first) : R;
        const bool has_row = grp < rows;
        const int i0 = upper ? n - 1 - first : first;  // row of group 0
        int i = 0, beg = 0, end = 0;
        if (has_row) {
            i = upper ? i0 - grp : i0 + grp;
            beg = ptr[i];
            end = ptr[i + 1];
        }
        int q0 = beg + sl;
        int c[E], v[E];
        unsigned live = 0, pend = 0, local = 0;  // local: dependency inside this ticket
        auto load_chunk = [&]() {
            live = pend = local = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int qq = q0 + e * W;
                c[e] = -1;
                v[e] = -1;
                if (qq < end) {
                    const int cc = idx[qq];
                    if (cc != i) {
                        c[e] = cc;
                        live |= 1u << e;
                        const int g2 = upper ? i0 - cc : cc - i0;  // owning group, if in ticket
                        if (g2 >= 0 && g2 < grp) local |= 1u << e;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((live & ~local) & (1u << e)) v[e] = ld_relaxed(lev + c[e]);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((live & (1u << e)) && v[e] < 0) pend |= 1u << e;
        };
        bool lane_done = q0 >= end;
        if (!lane_done) load_chunk();
        bool published = !has_row;
        int pub = -1;  // this group's level once published (same on all its lanes)
        int m = -1;
        long long waits = 0;
        unsigned ns = 32;
        while (true) {
            if (!lane_done && pend == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (live & (1u << e)) m = max(m, v[e]);
                q0 += W * E;
                if (q0 >= end) lane_done = true;
                else load_chunk();
            }
            const unsigned done = __ballot_sync(FULL, lane_done);
            const bool row_ready = (done & gmask) == gmask;
            const int tot = group_max<W>(m, FULL);
            if (row_ready && !published) {
                pub = tot + 1;
                if (sl == 0) {
                    st_relaxed(lev + i, pub);
                    local_max = max(local_max, pub);
                }
                published = true;
            }
            if (__all_sync(FULL, published)) break;
            // dependencies inside the ticket: read the owner's level by shuffle
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const bool want = (pend & local & (1u << e)) != 0;
                const int g2 = want ? (upper ? i0 - c[e] : c[e] - i0) : grp;
                const int got = __shfl_sync(FULL, pub, g2 * W);
                if (want && got >= 0) {
                    v[e] = got;
                    pend &= ~(1u << e);
                }
            }
            if (__any_sync(FULL, (pend & ~local) != 0)) {
                const unsigned far = pend & ~local;
                if (far) {
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (far & (1u << e)) v[e] = ld_relaxed(lev + c[e]);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if ((far & (1u << e)) && v[e] >= 0) pend &= ~(1u << e);
                }
                if (++waits >= sp.limit) {
                    if (far) {
                        report(status, i, kCodeTimeout);
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if (far & (1u << e)) v[e] = 0;
                        pend &= local;
                    }
                } else if (waits >= sp.hot) {
                    __nanosleep(ns);
                    ns = ns < sp.max_ns ? ns * 2 : sp.max_ns;
                }
            } else {
                waits = 0;
                ns = 32;
            }
        }
        t = __shfl_sync(FULL, tn, 0);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        local_max = max(local_max, __shfl_xor_sync(FULL, local_max, off));
    if (lane == 0 && local_max >= 0) atomicMax(nlev, local_max + 1);
}

template <int W>
static cudaError_t sweep_w(int n, const int* ptr, const int* idx, bool upper, int* lev,
                           int* ticket, int* nlev, unsigned long long* status, SpinPolicy sp,
                           int grid, int block, cudaStream_t s) {
    level_sweep_k<W><<<grid, block, 0, s>>>(n, ptr, idx, upper, lev, ticket, nlev, status, sp);
    return cudaGetLastError();
}

cudaError_t launch_level_sweep(int lanes, int n, const int* ptr, const int* idx, bool upper,
                               int* lev, int* ticket, int* nlev, unsigned long long* status,
                               SpinPolicy sp, int grid, int block, cudaStream_t s) {
    switch (lanes) {
        case 1: return sweep_w<1>(n, ptr, idx, upper, lev, ticket, nlev, status, sp, grid, block, s);
        case 2: return sweep_w<2>(n, ptr, idx, upper, lev, ticket, nlev, status, sp, grid, block, s);
        case 4: return sweep_w<4>(n, ptr, idx, upper, lev, ticket, nlev, status, sp, grid, block, s);
        case 8: return sweep_w<8>(n, ptr, idx, upper, lev, ticket, nlev, status, sp, grid, block, s);
        case 16: return sweep_w<16>(n, ptr, idx, upper, lev, ticket, nlev, status, sp, grid, block, s);
        case 32: return sweep_w<32>(n, ptr, idx, upper, lev, ticket, nlev, status, sp, grid, block, s);
        default: return cudaErrorInvalidValue;
    }
}

int level_sweep_blocks_per_sm(int lanes, int block) {
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (lanes) {
        case 1: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_sweep_k<1>, block, 0); break;
        case 2: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_sweep_k<2>, block, 0); break;
        case 4: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_sweep_k<4>, block, 0); break;
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_sweep_k<8>, block, 0); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_sweep_k<16>, block, 0); break;
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, level_sweep_k<32>, block, 0); break;
    }
    return (e == cudaSuccess && nb > 0) ? nb : 1;
}

// ------------------------------------------------------------ segment sweep
// Levels of the segment graph for the chained solve.  Segments are runs of
// R = 32/W consecutive positions in substitution order; a segment depends on
// the segments holding its rows' out-of-segment dependencies, and
//     slev(S) = 1 + max slev(segments S depends on)      (0 with none).
// Contiguous segments of a triangular matrix always form an acyclic graph
// and every dependency points to an earlier segment, so segments are swept
// in order by ticket, exactly as rows are in level_sweep_k; edges inside a
// segment are ignored.  slev[] starts at -1.
template <int W>
__global__ void segment_sweep_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                                int upper, int* slev, int* ticket, int* nslev,
                                unsigned long long* status, SpinPolicy sp) {
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const long long nseg = ((long long)n + R - 1) / R;
    int top = 0;  // highest slev + 1 this warp published
    int t = 0;
    if (lane == 0) t = atomicAdd(ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while (t < nseg) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(ticket, 1);
        const long long p0 = (long long)t * R;
        const long long pos = p0 + grp;
        int i = 0, beg = 0, end = 0;
        if (pos < n) {
            i = upper ? (int)(n - 1 - pos) : (int)pos;
            beg = ptr[i];
            end = ptr[i + 1];
        }
        int q0 = beg + sl;
        int c[E], v[E];
        unsigned live = 0, pend = 0;
        auto load_chunk = [&]() {
            live = pend = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int qq = q0 + e * W;
                c[e] = -1;
                v[e] = -1;
                if (qq < end) {
                    const int cc = idx[qq];
                    const long long cp = upper ? (long long)(n - 1 - cc) : (long long)cc;
                    if (cc != i && cp < p0) {  // out-of-segment dependency
                        c[e] = (int)(cp / R);
                        live |= 1u << e;
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (live & (1u << e)) v[e] = ld_relaxed(slev + c[e]);
#pragma unroll
            for (int e = 0; e < E; ++e)
                if ((live & (1u << e)) && v[e] < 0) pend |= 1u << e;
        };
        bool lane_done = q0 >= end;
        if (!lane_done) load_chunk();
        int m = -1;
        long long waits = 0;
        unsigned ns = 32;
        while (true) {
            if (!lane_done && pend == 0) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (live & (1u << e)) m = max(m, v[e]);
                q0 += W * E;
                if (q0 >= end) lane_done = true;
                else load_chunk();
            }
            if (__all_sync(FULL, lane_done)) break;
            if (__any_sync(FULL, !lane_done && pend == 0)) continue;
            if (pend) {
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if (pend & (1u << e)) v[e] = ld_relaxed(slev + c[e]);
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((pend & (1u << e)) && v[e] >= 0) pend &= ~(1u << e);
            }
            if (++waits >= sp.limit) {
                if (pend) {
                    report(status, i, kCodeTimeout);
#pragma unroll
                    for (int e = 0; e < E; ++e)
                        if (pend & (1u << e)) v[e] = 0;
                    pend = 0;
                }
                waits = 0;
            } else if (waits >= sp.hot) {
                __nanosleep(ns);
                ns = ns < sp.max_ns ? ns * 2 : sp.max_ns;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(FULL, m, off));
        if (lane == 0) st_relaxed(slev + t, m + 1);
        top = max(top, m + 2);
        t = __shfl_sync(FULL, tn, 0);
    }
    if (lane == 0 && top > 0) atomicMax(nslev, top);
}

cudaError_t launch_segment_sweep(int lanes, int n, const int* ptr, const int* idx, bool upper,
                                 int* slev, int* ticket, int* nslev, unsigned long long* status,
                                 SpinPolicy sp, int grid, int block, cudaStream_t s) {
#define SPTRSV_SEG(WW) \
    segment_sweep_k<WW><<<grid, block, 0, s>>>(n, ptr, idx, upper, slev, ticket, nslev, status, sp)
    switch (lanes) {
        case 1: SPTRSV_SEG(1); break;
        case 2: SPTRSV_SEG(2); break;
        case 4: SPTRSV_SEG(4); break;
        case 8: SPTRSV_SEG(8); break;
        case 16: SPTRSV_SEG(16); break;
        case 32: SPTRSV_SEG(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef SPTRSV_SEG
    return cudaGetLastError();
}

// ------------------------------------------------------------ histogram
// count[keys[e]] += 1, with lanes holding equal keys combined first.
__global__ void histogram_k(const int* __restrict__ keys, int m, int* count, int bins,
                            unsigned long long* status) {
    for (long long e0 = (long long)blockIdx.x * blockDim.x; e0 < m;
         e0 += (long long)gridDim.x * blockDim.x) {
        const long long e = e0 + threadIdx.x;
        const int lane = threadIdx.x & 31;
        int key = e < m ? keys[e] : -1 - lane;  // invalid lanes never match
        if (e < m && (key < 0 || key >= bins)) {
            report(status, (int)e, kCodeInternal);
            key = -1 - lane;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (key >= 0 && lane == __ffs(peers) - 1) atomicAdd(count + key, __popc(peers));
    }
}

cudaError_t launch_histogram(const int* keys, int m, int* count, int bins,
                             unsigned long long* status, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    long long g = ((long long)m + 255) / 256;
    if (g > 4096) g = 4096;
    histogram_k<<<(int)g, 256, 0, s>>>(keys, m, count, bins, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ exclusive scan
// Exclusive scan in three coalesced phases: every block sums its chunk
// (phase 1), one block scans the block sums (phase 2), every block scans its
// chunk tile by tile with the chunk's offset as the carry-in (phase 3).
constexpr int kScanThreads = 1024;
constexpr int kScanBlocks = 1024;  // phase 2 scans these sums in one block

__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        const int t = lane < nw ? warp_tot[lane] : 0;
        int wi = t;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < nw) warp_tot[lane] = wi - t;
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const int r = warp_tot[w] + incl - v;
    __syncthreads();  // warp_tot may be reused by the caller's next call
    return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_block_sums_k(const int* __restrict__ in,
                                                                 int m, long long chunk,
                                                                 int* sums) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < m ? lo + chunk : m;
    int s = 0;
    for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) s += in[e];
    block_exclusive_scan(s, warp_tot, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_sums_k(int* sums, int nb) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    const int v = threadIdx.x < nb ? sums[threadIdx.x] : 0;
    const int ex = block_exclusive_scan(v, warp_tot, &total);
    if (threadIdx.x < nb) sums[threadIdx.x] = ex;
    if (threadIdx.x == 0) sums[nb] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_chunks_k(const int* __restrict__ in,
                                                             int* out, int m, long long chunk,
                                                             const int* __restrict__ sums,
                                                             int nb) {
    __shared__ int warp_tot[32];
    __shared__ int total;
    const long long lo = (long long)blockIdx.x * chunk;
    const long long hi = lo + chunk < m ? lo + chunk : m;
    int carry = sums[blockIdx.x];
    for (long long base = lo; base < hi; base += blockDim.x) {
        const long long e = base + threadIdx.x;
        const int v = e < hi ? in[e] : 0;
        const int ex = block_exclusive_scan(v, warp_tot, &total);
        if (e < hi) out[e] = carry + ex;
        carry += total;
    }
    if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[m] = sums[nb];
}

// out[0..m]: exclusive prefix sums of in[0..m-1], out[m] = total (in and
// out must not overlap).  The block sums take at most kScanBlocks + 1 ints
// of stream-ordered scratch (setup paths only; never under capture).
cudaError_t launch_exclusive_scan(const int* in, int* out, int m, cudaStream_t s) {
    if (m <= 0) {
        return cudaMemsetAsync(out, 0, sizeof(int), s);
    }
    const long long per_block_min = kScanThreads;
    long long nb = ((long long)m + per_block_min - 1) / per_block_min;
    if (nb > kScanBlocks) nb = kScanBlocks;
    long long chunk = ((long long)m + nb - 1) / nb;
    chunk = (chunk + kScanThreads - 1) / kScanThreads * kScanThreads;
    nb = ((long long)m + chunk - 1) / chunk;
    int* sums = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(int) * (size_t)(nb + 1), s);
    if (e != cudaSuccess) return e;
    scan_block_sums_k<<<(int)nb, kScanThreads, 0, s>>>(in, m, chunk, sums);
    scan_sums_k<<<1, kScanThreads, 0, s>>>(sums, (int)nb);
    scan_chunks_k<<<(int)nb, kScanThreads, 0, s>>>(in, out, m, chunk, sums, (int)nb);
    e = cudaGetLastError();
    cudaError_t f = cudaFreeAsync(sums, s);
    return e != cudaSuccess ? e : f;
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort, 8-bit digits.  Per pass: per-tile digit counts,
// one exclusive scan over (digit, tile), then a stable scatter in which
// each warp ranks its lanes with __match_any_sync and warps are ordered
// through a shared-memory table.
constexpr int kRsThreads = 512;
constexpr int kRsTile = 8192;
constexpr int kRsWarps = kRsThreads / 32;

int radix_hist_entries(int m) {
    const int nb = (m + kRsTile - 1) / kRsTile;
    return 256 * (nb > 0 ? nb : 1);
}

__global__ void __launch_bounds__(kRsThreads) rs_hist_k(const int* __restrict__ keys, int m,
                                                        int shift, int* ghist, int nb) {
    __shared__ int h[256];
    for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
    __syncthreads();
    const long long t0 = (long long)blockIdx.x * kRsTile;
    const long long t1 = t0 + kRsTile < m ? t0 + kRsTile : m;
    for (long long e = t0 + threadIdx.x; e < t1; e += blockDim.x)
        atomicAdd(&h[(keys[e] >> shift) & 255], 1);
    __syncthreads();
    for (int t = threadIdx.x; t < 256; t += blockDim.x) ghist[t * nb + blockIdx.x] = h[t];
}

__global__ void __launch_bounds__(kRsThreads) rs_scatter_k(const int* __restrict__ kin,
                                                           const int* __restrict__ vin, int m,
                                                           int shift, const int* __restrict__ gofs,
                                                           int nb, int* kout, int* vout,
                                                           unsigned long long* status) {
    __shared__ int table[kRsWarps][256];
    __shared__ int base[256];
    __shared__ int total[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int t = threadIdx.x; t < 256; t += kRsThreads) base[t] = gofs[t * nb + blockIdx.x];
    const long long t0 = (long long)blockIdx.x * kRsTile;
    const long long t1 = t0 + kRsTile < m ? t0 + kRsTile : m;
    for (long long c0 = t0; c0 < t1; c0 += kRsThreads) {
        for (int t = threadIdx.x; t < kRsWarps * 256; t += kRsThreads) (&table[0][0])[t] = 0;
        __syncthreads();
        const long long e = c0 + threadIdx.x;
        const bool valid = e < t1;
        int key = 0, val = 0, d = 256 + lane;  // invalid lanes: a digit nobody else has
        if (valid) {
            key = kin[e];
            val = vin ? vin[e] : (int)e;
            d = (key >> shift) & 255;
        }
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && lane == __ffs(peers) - 1) table[w][d] = __popc(peers);
        __syncthreads();
        if (threadIdx.x < 256) {
            int run = 0;
            for (int ww = 0; ww < kRsWarps; ++ww) {
                const int c = table[ww][threadIdx.x];
                table[ww][threadIdx.x] = run;
                run += c;
            }
            total[threadIdx.x] = run;
        }
        __syncthreads();
        if (valid) {
            const int pos = base[d] + table[w][d] + rank;
            if (pos >= 0 && pos < m) {
                kout[pos] = key;
                vout[pos] = val;
            } else {
                report(status, (int)e, kCodeInternal);
            }
        }
        __syncthreads();
        if (threadIdx.x < 256) base[threadIdx.x] += total[threadIdx.x];
    }
}

__global__ void iota_k(int* out, int m) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (long long)gridDim.x * blockDim.x)
        out[e] = (int)e;
}

cudaError_t launch_iota(int* out, int m, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    long long g = ((long long)m + 255) / 256;
    if (g > 4096) g = 4096;
    iota_k<<<(int)g, 256, 0, s>>>(out, m);
    return cudaGetLastError();
}

cudaError_t radix_sort_values(const int* keys_in, const int* vals_in, int m, int bits,
                              int* vals_out, int* k_a, int* v_a, int* k_b, int* v_b, int* hist,
                              int* hist_scan, unsigned long long* status, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    const int passes = (bits + 7) / 8;
    if (passes == 0) {
        if (vals_in) return cudaMemcpyAsync(vals_out, vals_in, sizeof(int) * (size_t)m,
                                            cudaMemcpyDeviceToDevice, s);
        return launch_iota(vals_out, m, s);
    }
    const int nb = (m + kRsTile - 1) / kRsTile;
    const int* kin = keys_in;
    const int* vin = vals_in;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        int* kout = (pass & 1) ? k_b : k_a;
        int* vout = (pass == passes - 1) ? vals_out : ((pass & 1) ? v_b : v_a);
        rs_hist_k<<<nb, kRsThreads, 0, s>>>(kin, m, shift, hist, nb);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = launch_exclusive_scan(hist, hist_scan, 256 * nb, s);
        if (e != cudaSuccess) return e;
        rs_scatter_k<<<nb, kRsThreads, 0, s>>>(kin, vin, m, shift, hist_scan, nb, kout, vout,
                                                 status);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        kin = kout;
        vin = vout;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------ transpose helpers
__global__ void row_of_entries_k(int n, const int* __restrict__ ptr, int* rowof) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int end = ptr[i + 1];
        for (int q = ptr[i]; q < end; ++q) rowof[q] = (int)i;
    }
}

cudaError_t launch_row_of_entries(int n, const int* ptr, int* rowof, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 4096) g = 4096;
    row_of_entries_k<<<(int)g, 256, 0, s>>>(n, ptr, rowof);
    return cudaGetLastError();
}

__global__ void gather_k(const int* __restrict__ src, int src_len,
                         const int* __restrict__ index, int m, int* out,
                         unsigned long long* status) {
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (long long)gridDim.x * blockDim.x) {
        const int j = index[e];
        if (j >= 0 && j < src_len) {
            out[e] = src[j];
        } else {
            out[e] = -1;
            report(status, (int)e, kCodeInternal);
        }
    }
}

cudaError_t launch_gather(const int* src, int src_len, const int* index, int m, int* out,
                          unsigned long long* status, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    long long g = ((long long)m + 255) / 256;
    if (g > 8192) g = 8192;
    gather_k<<<(int)g, 256, 0, s>>>(src, src_len, index, m, out, status);
    return cudaGetLastError();
}

// ------------------------------------------------------------ inverse permutation
// ipos[jlev[k]] = k: the position of every row in level order.
__global__ void inverse_perm_k(const int* __restrict__ perm, int n, int* ipos) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x)
        ipos[perm[k]] = (int)k;
}

cudaError_t launch_inverse_perm(const int* perm, int n, int* ipos, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 4096) g = 4096;
    inverse_perm_k<<<(int)g, 256, 0, s>>>(perm, n, ipos);
    return cudaGetLastError();
}

// ------------------------------------------------------------ level-set check
__global__ void verify_levels_k(int n, int nlev, const int* __restrict__ lev,
                                const int* __restrict__ ilev, const int* __restrict__ jlev,
                                unsigned long long* status) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && (ilev[0] != 0 || ilev[nlev] != n))
        report(status, 0, kCodeInternal);
    for (long long kk = (long long)blockIdx.x * blockDim.x + threadIdx.x; kk < n;
         kk += (long long)gridDim.x * blockDim.x) {
        const int k = (int)kk;
        const int i = jlev[k];
        if (i < 0 || i >= n) {
            report(status, k, kCodeInternal);
            continue;
        }
        const int m = lev[i];
        if (m < 0 || m >= nlev || k < ilev[m] || k >= ilev[m + 1]) {
            report(status, k, kCodeInternal);
            continue;
        }
        if (k > ilev[m]) {
            const int prev = jlev[k - 1];
            if (prev >= i) report(status, k, kCodeInternal);
        }
    }
}

cudaError_t launch_verify_levels(int n, int nlev, const int* lev, const int* ilev,
                                 const int* jlev, unsigned long long* status, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 4096) g = 4096;
    verify_levels_k<<<(int)g, 256, 0, s>>>(n, nlev, lev, ilev, jlev, status);
    return cudaGetLastError();
}

// Self-check of the segment levels of the chained solve: every
// out-of-segment dependency of a row lies in a segment of strictly lower
// level (the chained solve's deadlock freedom rests on it).
__global__ void verify_segments_k(int n, int R, const int* __restrict__ ptr,
                                  const int* __restrict__ idx, int upper,
                                  const int* __restrict__ slev, int nslev,
                                  unsigned long long* status) {
    for (long long ii = (long long)blockIdx.x * blockDim.x + threadIdx.x; ii < n;
         ii += (long long)gridDim.x * blockDim.x) {
        const int i = (int)ii;
        const long long pos = upper ? (long long)(n - 1 - i) : ii;
        const long long seg = pos / R;
        const int own = slev[seg];
        if (own < 0 || own >= nslev) {
            report(status, i, kCodeInternal);
            continue;
        }
        for (int q = ptr[i]; q < ptr[i + 1]; ++q) {
            const int c = idx[q];
            const long long cp = upper ? (long long)(n - 1 - c) : (long long)c;
            if (c != i && cp / R != seg && slev[cp / R] >= own) report(status, i, kCodeInternal);
        }
    }
}

cudaError_t launch_verify_segments(int n, int R, const int* ptr, const int* idx, bool upper,
                                   const int* slev, int nslev, unsigned long long* status,
                                   cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 4096) g = 4096;
    verify_segments_k<<<(int)g, 256, 0, s>>>(n, R, ptr, idx, upper, slev, nslev, status);
    return cudaGetLastError();
}

}  // namespace sptrsv
