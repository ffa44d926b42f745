// Part-ordered copy for the partitioned solve (SPTRSV_ALGO_SELF_PARTITIONED):
// level-scheduled order inside a part of consecutive rows.
//
// Parts are runs of consecutive rows in order of substitution (ascending for
// a lower system, descending for an upper one), so every dependency of a
// part lies in the part itself or in an earlier part of the same run.  The
// copy lists the parts one after another and, inside a part, its rows by
// level (Sec. 4.1), then row; every column index is renumbered to its
// position in that order.  A dependency then points to an earlier position,
// one inside the part to a row of a lower level of the same part.  The
// blocked self-scheduled kernel (solve_blocked.cu) runs on this copy with one
// part per tile: a thread block holds its part's unknowns in shared memory,
// where dependencies inside the part are served, and waits for earlier parts
// through the published values as in Alg. 3.  On a structured grid in natural
// order a part is a slab of whole grid lines, so the dependency hops along
// the lines stay in shared memory and only the hops between slabs go through
// L2; with levels as the order inside a part its rows are taken as they
// become ready.
//
// How the rows are cut into parts.  The substitution order is first split
// where the matrix decouples: position t starts an independent block when no
// row at or after t depends on a row before t (a block-diagonal batch of
// systems decouples at every system boundary).  These boundaries come from
// one difference array: a row at position u whose farthest dependency is at
// position f < u covers the positions f+1 .. u, and the positions no row
// covers are the block starts.  A block longer than half the part size S is
// cut into ceil(len/S) pieces of balanced length; shorter blocks that start
// in the same window of S/2 positions share one part (so a part never holds
// more than S rows).  A part never straddles two blocks unless all of them
// fit in it whole.  The parts are then handed out latest start first: a
// part's key is the level at which it must start at the latest for its
// block to finish with the deepest one -- the block's slack (deepest level
// of the matrix minus the block's own depth) plus the piece's share of the
// block's levels (piece index times levels per piece) -- and parts with
// equal keys go in order of substitution.  Keys do not decrease along a
// block's pieces, so every part still depends only on parts handed out
// before it.  The pieces of the deepest systems of a batch are taken as the
// frontier reaches them, and short systems, which have slack, fill the
// blocks in between; handing out every system's first piece before any
// second piece (the previous order) left the deepest system's later pieces
// queued behind hundreds of short systems (batch of 512: 5.06 -> 4.64 ms).
#include "internal.h"

namespace sptrsv {

namespace {

int grid_for(long long m) {
    long long g = (m + 255) / 256;
    if (g > 8192) g = 8192;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

// diff[f + 1] += 1 and diff[t + 1] -= 1 for the row at substitution position
// t whose farthest dependency sits at position f < t.
__global__ void part_spans_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                             int upper, int* diff) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (long long)gridDim.x * blockDim.x) {
        const int beg = ptr[r], end = ptr[r + 1];
        if (beg >= end) continue;
        // columns ascend inside a row: the farthest dependency is the first
        // entry of a lower row and the last entry of an upper one
        const int c = upper ? idx[end - 1] : idx[beg];
        if (c == (int)r) continue;  // only the diagonal
        const long long t = upper ? n - 1 - r : r;
        const long long f = upper ? n - 1 - c : c;
        atomicAdd(diff + f + 1, 1);
        atomicAdd(diff + t + 1, -1);
    }
}

// flag[t] = 1 where no dependency span covers t (t = 0 always): a block start.
__global__ void block_flags_k(int n, const int* __restrict__ cover, int* flag) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        flag[t] = (t == 0 || cover[t + 1] == 0) ? 1 : 0;
}

// start[scan[t]] = t where flag[t]; start[scan[n]] = n.
__global__ void flag_scatter_k(int n, const int* __restrict__ flag, const int* __restrict__ scan,
                               int* start) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        if (flag[t]) start[scan[t]] = (int)t;
    if (blockIdx.x == 0 && threadIdx.x == 0) start[scan[n]] = n;
}

// depth[b] = largest level of the rows of block b (an atomic max per warp
// when its lanes hold one block, which is the common case).
__global__ void block_depth_k(int n, int upper, const int* __restrict__ lev,
                              const int* __restrict__ bscan, int* depth) {
    for (long long t0 = (long long)blockIdx.x * blockDim.x; t0 < n;
         t0 += (long long)gridDim.x * blockDim.x) {
        const long long t = t0 + threadIdx.x;
        const bool in = t < n;
        const int b = in ? bscan[t + 1] - 1 : -1;
        const int l = in ? lev[upper ? n - 1 - t : t] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int m = __reduce_max_sync(peers, l);
        if (in && (threadIdx.x & 31) == __ffs(peers) - 1) atomicMax(depth + b, m);
    }
}

// flag[t] = 1 where a part starts: at the pieces of a long block (longer than
// h = S/2, cut into ceil(len/S) balanced pieces) and at a short block that
// follows a long one or starts in another window of h positions than the
// short block before it.
__global__ void part_flags_k(int n, int S, const int* __restrict__ bscan,
                             const int* __restrict__ bstart, int* flag) {
    const long long h = S / 2 > 0 ? S / 2 : 1;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = bscan[t + 1] - 1;
        const long long st = bstart[b], len = bstart[b + 1] - st;
        int f;
        if (len > h) {
            const long long np = (len + S - 1) / S;
            f = (t == st || (t - st) * np / len != (t - 1 - st) * np / len) ? 1 : 0;
        } else if (t != st) {
            f = 0;
        } else if (b == 0) {
            f = 1;
        } else {
            const long long pst = bstart[b - 1];
            f = (st - pst > h || st / h != pst / h) ? 1 : 0;
        }
        flag[t] = f;
    }
}

// key[p] = deepest level minus the depth of the block part p starts in, so
// that an ascending stable sort hands the deepest blocks out first.
__global__ void part_depth_keys_k(int np, int maxdepth, const int* __restrict__ pstart,
                                  const int* __restrict__ bscan, const int* __restrict__ depth,
                                  int* key) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x)
        key[p] = maxdepth - depth[bscan[pstart[p] + 1] - 1];
}

// piece[p] = index of part p among the parts of its block (0 for the first).
__global__ void part_piece_k(int np, const int* __restrict__ pstart,
                             const int* __restrict__ bscan, const int* __restrict__ bstart,
                             const int* __restrict__ pscan, int* piece) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = bscan[pstart[p] + 1] - 1;
        piece[p] = (int)p - (pscan[bstart[b] + 1] - 1);
    }
}

// key[p] = the estimated latest level at which part p can start: its
// block's slack (deepest level minus the block's depth) plus its piece's
// share of the block's levels (piece index times levels per piece).  Keys do
// not decrease along a block's pieces, so a stable sort keeps them in order.
__global__ void part_alap_keys_k(int np, int maxdepth, const int* __restrict__ pstart,
                                 const int* __restrict__ bscan, const int* __restrict__ bstart,
                                 const int* __restrict__ pscan, const int* __restrict__ depth,
                                 const int* __restrict__ piece, int* key) {
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
         p += (long long)gridDim.x * blockDim.x) {
        const int b = bscan[pstart[p] + 1] - 1;
        const int d = depth[b];
        const int first = pscan[bstart[b] + 1] - 1;  // the block's first part
        const int cnt = pscan[bstart[b + 1]] - first;  // parts starting in the block
        const long long share = cnt > 1 ? (long long)piece[p] * (d + 1) / cnt : 0;
        key[p] = (maxdepth - d) + (int)share;
    }
}

// size[r] = rows of the part handed out r-th; atomic max of the sizes.
__global__ void part_sizes_k(int np, const int* __restrict__ horder,
                             const int* __restrict__ pstart, int* size, int* maxsize) {
    int m = 0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < np;
         r += (long long)gridDim.x * blockDim.x) {
        const int p = horder[r];
        const int s = pstart[p + 1] - pstart[p];
        size[r] = s;
        m = max(m, s);
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) atomicMax(maxsize, m);
}

// key[k] = hand-out rank of the part of row jlev[k].
__global__ void row_part_keys_k(int n, const int* __restrict__ jlev, int upper,
                                const int* __restrict__ pscan, const int* __restrict__ prank,
                                int* key) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = jlev[k];
        const long long t = upper ? n - 1 - i : i;
        key[k] = prank[pscan[t + 1] - 1];
    }
}

#define SPTRSV_LAUNCH(kernel, m, ...)                        \
    do {                                                     \
        kernel<<<grid_for(m), 256, 0, s>>>(__VA_ARGS__);     \
        cudaError_t _e = cudaGetLastError();                 \
        if (_e != cudaSuccess) return _e;                    \
    } while (0)

cudaError_t launch_part_spans(int n, const int* ptr, const int* idx, bool upper, int* diff,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(part_spans_k, n, n, ptr, idx, upper ? 1 : 0, diff);
    return cudaSuccess;
}

cudaError_t launch_block_flags(int n, const int* cover, int* flag, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(block_flags_k, n, n, cover, flag);
    return cudaSuccess;
}

cudaError_t launch_flag_scatter(int n, const int* flag, const int* scan, int* start,
                                cudaStream_t s) {
    SPTRSV_LAUNCH(flag_scatter_k, n, n, flag, scan, start);
    return cudaSuccess;
}

cudaError_t launch_block_depth(int n, bool upper, const int* lev, const int* bscan, int* depth,
                               cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(block_depth_k, n, n, upper ? 1 : 0, lev, bscan, depth);
    return cudaSuccess;
}

cudaError_t launch_part_flags(int n, int S, const int* bscan, const int* bstart, int* flag,
                              cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(part_flags_k, n, n, S, bscan, bstart, flag);
    return cudaSuccess;
}

cudaError_t launch_part_depth_keys(int np, int maxdepth, const int* pstart, const int* bscan,
                                   const int* depth, int* key, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(part_depth_keys_k, np, np, maxdepth, pstart, bscan, depth, key);
    return cudaSuccess;
}

cudaError_t launch_part_piece(int np, const int* pstart, const int* bscan, const int* bstart,
                              const int* pscan, int* piece, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(part_piece_k, np, np, pstart, bscan, bstart, pscan, piece);
    return cudaSuccess;
}

cudaError_t launch_part_alap_keys(int np, int maxdepth, const int* pstart, const int* bscan,
                                  const int* bstart, const int* pscan, const int* depth,
                                  const int* piece, int* key, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(part_alap_keys_k, np, np, maxdepth, pstart, bscan, bstart, pscan, depth, piece,
                  key);
    return cudaSuccess;
}

cudaError_t launch_part_sizes(int np, const int* horder, const int* pstart, int* size,
                              int* maxsize, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(part_sizes_k, np, np, horder, pstart, size, maxsize);
    return cudaSuccess;
}

cudaError_t launch_row_part_keys(int n, const int* jlev, bool upper, const int* pscan,
                                 const int* prank, int* key, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    SPTRSV_LAUNCH(row_part_keys_k, n, n, jlev, upper ? 1 : 0, pscan, prank, key);
    return cudaSuccess;
}

#undef SPTRSV_LAUNCH

}  // namespace sptrsv
