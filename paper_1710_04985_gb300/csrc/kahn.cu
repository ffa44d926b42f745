// Level analysis by Kahn's topological sort (Sec. 4.4.1), the setup the
// paper runs on the GPU, kept beside the sync-free sweep of analysis.cu for
// comparison (sptrsv_reanalyze).
//
// Kahn's algorithm peels the dependency DAG one level at a time: the roots
// (rows with no pending dependency) form level 0; removing a level's rows
// and their outgoing edges exposes the next level's roots.  Outgoing edges of
// row i are the entries of column i, read as row i of the CSR of the
// transpose (the DEP/TRANS steps of Table 1), and count(r) holds the
// dependencies of row r not yet removed.
//
// Two drivers:
//  * host loop, as in the paper: one launch per level and one device-to-host
//    copy of the queue end after it, so the host knows the next frontier;
//  * persistent: one cooperative launch sweeps every level, the frontiers
//    separated by a grid-wide barrier instead of a kernel boundary and a
//    copy.  The barrier is a monotone arrival counter with bounded waits:
//    past the spin limit a block records SPTRSV_ERR_TIMEOUT and stops, so the
//    launch always ends (a cooperative launch keeps every block resident, so
//    the limit is reached only if a block died).
// Both produce lev[] (0-based, the level at which each row became a root)
// and the level count; the level sets are then built from lev[] exactly as
// after the sweep, so every method gives the same ilev/jlev.
#include "internal.h"

namespace sptrsv {

// Level 0: count = count0; rows without dependencies are roots.
__global__ void kahn_roots_k(int n, const int* __restrict__ count0, int* count, int* lev,
                             int* queue, int* qend) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const int c = count0[r];
        count[r] = c;
        if (c == 0) {
            lev[r] = 0;
            queue[atomicAdd(qend, 1)] = (int)r;
        } else {
            lev[r] = -1;
        }
    }
}

cudaError_t launch_kahn_roots(int n, const int* count0, int* count, int* lev, int* queue,
                              int* qend, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 65535) g = 65535;
    kahn_roots_k<<<(int)g, 256, 0, s>>>(n, count0, count, lev, queue, qend);
    return cudaGetLastError();
}

// Removes the frontier queue[first, last) (rows of level `level`): a warp
// per frontier row, its lanes over the row's outgoing edges; a dependent
// whose count drops to zero becomes a root of level + 1 and is appended at
// *qend.  A queue entry past n (impossible for a valid pattern) is reported.
__device__ __forceinline__ void kahn_remove(const int* __restrict__ dptr,
                                            const int* __restrict__ didx, int* count, int* lev,
                                            int* queue, int* qend, int n, int i, int level,
                                            int lane, unsigned long long* status) {
    const int beg = dptr[i], end = dptr[i + 1];
    for (int q = beg + lane; q < end; q += 32) {
        const int r = didx[q];
        if (r == i) continue;
        if (atomicSub(count + r, 1) == 1) {
            lev[r] = level + 1;
            const int at = atomicAdd(qend, 1);
            if (at < n) queue[at] = r;
            else report(status, r, kCodeInternal);
        }
    }
}

__global__ void kahn_level_k(const int* __restrict__ dptr, const int* __restrict__ didx,
                             int* count, int* lev, int* queue, int* qend, int n, int first,
                             int last, int level, unsigned long long* status) {
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long w = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5);
         first + w < last; w += warps)
        kahn_remove(dptr, didx, count, lev, queue, qend, n, __ldcg(queue + first + w), level,
                    lane, status);
}

cudaError_t launch_kahn_level(const int* dptr, const int* didx, int* count, int* lev, int* queue,
                              int* qend, int n, int first, int last, int level,
                              unsigned long long* status, int max_grid, cudaStream_t s) {
    const long long rows = (long long)last - first;
    if (rows <= 0) return cudaSuccess;
    long long g = (rows + 7) / 8;  // 8 warps per 256-thread block
    if (g > max_grid) g = max_grid;
    kahn_level_k<<<(int)g, 256, 0, s>>>(dptr, didx, count, lev, queue, qend, n, first, last,
                                        level, status);
    return cudaGetLastError();
}

// Grid-wide barrier for a cooperative launch: every block adds one arrival
// per barrier to a 64-bit counter (zero at launch) and waits until the
// counter reaches blocks * generation.  Release/acquire order the frontier
// writes of one generation before the reads of the next.  Returns false if
// the wait ran past the limit (then SPTRSV_ERR_TIMEOUT is recorded).
__device__ __forceinline__ bool grid_barrier(unsigned long long* arrivals,
                                             unsigned long long target, long long limit,
                                             unsigned long long* status, int row) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(arrivals) : "memory");
        long long spins = 0;
        while (true) {
            unsigned long long v;
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(arrivals)
                         : "memory");
            if (v >= target) break;
            if (++spins >= limit) {
                report(status, row, kCodeTimeout);
                ok = 0;
                break;
            }
            if (spins > 64) __nanosleep(64);
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Removes the frontier queue[base, base + size) of level `level` with the
// warps [w0, w0 + nw): a warp per frontier row, its lanes over the row's
// outgoing edges; roots of level + 1 are counted in *tail and stored after
// the frontier.  Queue entries may have been written by other SMs: they are
// read from L2 (__ldcg), never from a stale L1 line.
__device__ __forceinline__ void kahn_frontier(const int* __restrict__ dptr,
                                              const int* __restrict__ didx, int* count, int* lev,
                                              int* queue, int* tail, int n, long long base,
                                              int size, int level, long long w0, long long nw,
                                              int lane, unsigned long long* status) {
    int* next = queue + base + size;
    for (long long w = w0; w < size; w += nw) {
        const int i = __ldcg(queue + base + w);
        const int beg = dptr[i], end = dptr[i + 1];
        for (int q = beg + lane; q < end; q += 32) {
            const int r = didx[q];
            if (r == i) continue;
            if (atomicSub(count + r, 1) == 1) {
                lev[r] = level + 1;
                const int at = atomicAdd(tail, 1);
                if (base + size + at < n) next[at] = r;
                else report(status, r, kCodeInternal);
            }
        }
    }
}

// Persistent driver.  The frontier of level L is queue[base_L, base_L +
// size_L); its removal appends the roots of level L + 1 right after it.
// Level sizes live in three rotating counters cnt[L % 3]: the value read
// after a barrier must not move while slower readers still read it, so the
// roots of level L + 1 are counted in cnt[(L+1) % 3] (not in the one being
// read), and block 0 clears cnt[(L+2) % 3] at the start of level L: every
// reader read that counter (size of level L - 1) before the barrier that
// opened level L, and nobody appends to it before the next one.
//
// Wide levels run on the whole grid, one grid barrier each.  A level of at
// most `narrow` rows runs on block 0 alone, which keeps going through
// consecutive narrow levels separated only by block barriers (no grid-wide
// step) and then publishes (base, size, level) in ctl[0..2]; the other
// blocks meanwhile wait at the grid barrier that closes the run.  A run
// opens with one more grid barrier, after which every block has read the
// size it starts from, so block 0 may clear and reuse that counter.  Deep,
// narrow dependency graphs thus cost a block barrier per level, not a grid
// barrier.  cnt[0] holds the roots queued by kahn_roots_k; cnt[1], cnt[2]
// start at zero.  Writes the level count and cnt[3] = rows leveled.
constexpr int kNarrowRun = 4096;

__global__ void kahn_persistent_k(const int* __restrict__ dptr, const int* __restrict__ didx,
                                  int* count, int* lev, int* queue, int* cnt, int* ctl, int n,
                                  int narrow, int probe_level, int probe_min_avg,
                                  unsigned long long* arrivals, int* nlev_out,
                                  unsigned long long* status, long long limit) {
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long wid = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5);
    const int bwarps = blockDim.x >> 5, bwid = threadIdx.x >> 5;
    unsigned long long gen = 0;
    long long base = 0;
    int size = *(volatile int*)cnt;  // roots, queued before this launch
    int level = 0;
    // Level at which the next probe is taken (0: none left).
    int next_probe = probe_level > 0 ? probe_level : 0;
    bool postponed = false;
    while (size > 0) {
        // Early exit for deep, narrow graphs (a grid barrier per level costs
        // more there than the sweep): every block sees the same (base, size,
        // level) here, so all of them decide alike.  Levels that are still
        // widening (the current one at least 1.5 times the average so far)
        // get one second look at four times the level, which then asks for
        // a 1.5 times larger average.
        if (next_probe > 0 && level >= next_probe) {
            next_probe = 0;
            const long long need = postponed ? (3ll * probe_min_avg) / 2 : probe_min_avg;
            if (base < (long long)level * need) {
                if (!postponed && 2ll * size * level >= 3ll * base) {
                    postponed = true;
                    next_probe = 4 * level;
                } else {
                    if (blockIdx.x == 0 && threadIdx.x == 0) *nlev_out = -1;
                    return;
                }
            }
        }
        if (size <= narrow) {
            // Every block must have read `size` (the counter of the grid
            // barrier just passed) before block 0 runs ahead: its next levels
            // clear and reuse that counter.  One extra grid barrier per run.
            ++gen;
            if (!grid_barrier(arrivals, gen * gridDim.x, limit, status, level)) return;
            if (blockIdx.x == 0) {
                // at most kNarrowRun levels per run, so the other blocks' wait
                // at the closing barrier stays far below its spin limit; a run
                // also stops at the probe level so that the probe is taken
                for (int run = 0; run < kNarrowRun && size > 0 && size <= narrow &&
                                   (next_probe == 0 || level < next_probe);
                     ++run) {
                    if (threadIdx.x == 0) cnt[(level + 2) % 3] = 0;
                    __syncthreads();
                    int* tail = cnt + (level + 1) % 3;
                    kahn_frontier(dptr, didx, count, lev, queue, tail, n, base, size, level, bwid,
                                  bwarps, lane, status);
                    __syncthreads();  // every append of this level has been performed
                    int nsz;
                    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(nsz) : "l"(tail)
                                 : "memory");
                    __syncthreads();  // read by all before the next level appends
                    base += size;
                    size = nsz;
                    ++level;
                }
                if (threadIdx.x == 0) {
                    ctl[0] = (int)base;
                    ctl[1] = size;
                    ctl[2] = level;
                }
            }
            ++gen;
            if (!grid_barrier(arrivals, gen * gridDim.x, limit, status, level)) return;
            int st[3];
#pragma unroll
            for (int k = 0; k < 3; ++k)
                asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(st[k]) : "l"(ctl + k)
                             : "memory");
            base = st[0];
            size = st[1];
            level = st[2];
            continue;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(level + 2) % 3] = 0;
        int* tail = cnt + (level + 1) % 3;
        kahn_frontier(dptr, didx, count, lev, queue, tail, n, base, size, level, wid, warps, lane,
                      status);
        ++gen;
        if (!grid_barrier(arrivals, gen * gridDim.x, limit, status, level)) return;
        int nsz;
        asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(nsz) : "l"(tail) : "memory");
        base += size;
        size = nsz;
        ++level;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *nlev_out = level;
        cnt[3] = (int)base;  // rows leveled, checked by the host
    }
}

int kahn_persistent_blocks_per_sm(int block) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kahn_persistent_k, block, 0) !=
            cudaSuccess ||
        nb < 1)
        return 1;
    return nb;
}

cudaError_t launch_kahn_persistent(const int* dptr, const int* didx, int* count, int* lev,
                                   int* queue, int* cnt, int* ctl, int n, int narrow,
                                   int probe_level, int probe_min_avg,
                                   unsigned long long* arrivals, int* nlev_out,
                                   unsigned long long* status, long long limit, int grid,
                                   int block, cudaStream_t s) {
    void* args[] = {(void*)&dptr,        (void*)&didx,          (void*)&count,
                    (void*)&lev,         (void*)&queue,         (void*)&cnt,
                    (void*)&ctl,         (void*)&n,             (void*)&narrow,
                    (void*)&probe_level, (void*)&probe_min_avg, (void*)&arrivals,
                    (void*)&nlev_out,    (void*)&status,        (void*)&limit};
    return cudaLaunchCooperativeKernel((const void*)kahn_persistent_k, dim3(grid), dim3(block),
                                       args, 0, s);
}

}  // namespace sptrsv
