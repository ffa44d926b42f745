// Part-ordered copy for the partitioned solve (SPTRSV_ALGO_SELF_PARTITIONED):
// level-scheduled order inside a part of consecutive rows, parts in order of
// substitution.
//
// The rows are cut into parts of S consecutive rows (ascending for a lower
// system, descending for an upper one), so every dependency of a part lies
// in the part itself or in an earlier part.  The copy lists the parts one
// after another and, inside a part, its rows by level (Sec. 4.1), then row;
// every column index is renumbered to its position in that order.  A
// dependency then points to an earlier position, one inside the part to a
// row of a lower level of the same part.  The blocked self-scheduled kernel
// (solve_blocked.cu) runs on this copy with one part per tile: a thread
// block holds its part's unknowns in shared memory, where dependencies
// inside the part are served, and waits for earlier parts through the
// published values as in Alg. 3.  On a structured grid in natural order a
// part is a slab of whole grid lines, so the dependency hops along the lines
// stay in shared memory and only the hops between slabs go through L2; with
// levels as the order inside a part its rows are taken as they become ready.
#include "internal.h"

namespace sptrsv {

__global__ void part_keys_k(int n, const int* __restrict__ jlev, int S, int upper, int* key) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = jlev[k];
        key[k] = upper ? (n - 1 - i) / S : i / S;
    }
}

cudaError_t launch_part_keys(int n, const int* jlev, int S, bool upper, int* key,
                             cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 65535) g = 65535;
    part_keys_k<<<(int)g, 256, 0, s>>>(n, jlev, S, upper ? 1 : 0, key);
    return cudaGetLastError();
}

}  // namespace sptrsv
