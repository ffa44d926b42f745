// Level-ordered copy of a triangular pattern for SPTRSV_ALGO_SELF_PERMUTED.
//
// Sec. 4.3 (remark 2) observes that warps with consecutive indices do not
// work on consecutive unknowns when rows are taken in level order, and that
// preordering the matrix by level would restore that locality.  This file
// builds that preordering without touching the caller's arrays: position k
// of the level order jlev (Sec. 4.1) becomes row k of a copy whose entries
// are those of row jlev[k] in fold order -- a lower row's in their stored
// order, an upper row's reversed, so that every row is folded farthest
// dependency first (its diagonal then comes last) -- with every column index
// j replaced by the position ipos[j] of unknown j in jlev and the value
// copied beside it.  Dependencies then point to earlier positions (their
// levels are lower), a warp's rows are contiguous in memory, and the
// unknowns a level waits on are a contiguous run of the previous level.
#include "internal.h"

namespace sptrsv {

__global__ void ordered_lengths_k(int n, const int* __restrict__ ptr,
                                  const int* __restrict__ jlev, int* lens) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int i = jlev[k];
        lens[k] = ptr[i + 1] - ptr[i];
    }
}

cudaError_t launch_ordered_lengths(int n, const int* ptr, const int* jlev, int* lens,
                                   cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 65535) g = 65535;
    ordered_lengths_k<<<(int)g, 256, 0, s>>>(n, ptr, jlev, lens);
    return cudaGetLastError();
}

// One warp per position k; lanes stride over the row's entries, so long rows
// are copied with coalesced loads and stores; rev stores them last to first
// (an upper row: the fold order of every form).  pidx == nullptr refreshes the
// values only.  diag >= 0 (a matrix with a stored, used diagonal; 1: the
// diagonal is a row's first entry, 0: its last) stores the row pre-scaled
// as the self-scheduled kernels use it: 1/d(i) in the diagonal's slot and
// a_ij * (1/d(i)) for the other entries.  The kernels then skip the
// division and the scaling, and since both are the same IEEE operations
// they would do themselves, the results stay bitwise those of the unscaled
// form.
template <typename T>
__global__ void permute_rows_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                               const int* __restrict__ vmap, const T* __restrict__ vals,
                               const int* __restrict__ jlev, const int* __restrict__ ipos,
                               const int* __restrict__ pptr, int* pidx, T* pvals, int diag,
                               int rev) {
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long k = (((long long)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); k < n;
         k += warps) {
        const int i = jlev[k];
        const int beg = ptr[i], len = ptr[i + 1] - beg;
        const int out = pptr[k];
        T dinv = T(1);
        int qd = -1;
        if (diag >= 0 && len > 0) {
            qd = diag ? beg : beg + len - 1;
            dinv = T(1) / vals[vmap ? vmap[qd] : qd];
        }
        for (int e = lane; e < len; e += 32) {
            const int q = beg + e;
            const int at = out + (rev ? len - 1 - e : e);
            if (pidx) pidx[at] = ipos[idx[q]];
            const T v = vals[vmap ? vmap[q] : q];
            pvals[at] = diag < 0 ? v : (q == qd ? dinv : v * dinv);
        }
    }
}

cudaError_t launch_permute_rows(bool f64, int n, const int* ptr, const int* idx, const int* vmap,
                                const void* vals, const int* jlev, const int* ipos,
                                const int* pptr, int* pidx, void* pvals, int grid,
                                cudaStream_t s, int diag, bool rev) {
    if (n <= 0) return cudaSuccess;
    long long want = ((long long)n + 7) / 8;  // 8 warps of 256 threads per block
    int g = (int)(want < grid ? want : grid);
    if (g < 1) g = 1;
    if (f64)
        permute_rows_k<double><<<g, 256, 0, s>>>(n, ptr, idx, vmap, (const double*)vals, jlev,
                                                ipos, pptr, pidx, (double*)pvals, diag, rev);
    else
        permute_rows_k<float><<<g, 256, 0, s>>>(n, ptr, idx, vmap, (const float*)vals, jlev,
                                               ipos, pptr, pidx, (float*)pvals, diag, rev);
    return cudaGetLastError();
}

// Self-check of the copy: every entry of position k other than k itself
// names an earlier position (so the ticket order stays deadlock-free), and
// pptr is nondecreasing.  A failure is a library bug, reported as internal.
__global__ void verify_permuted_k(int n, const int* __restrict__ pptr,
                                  const int* __restrict__ pidx, unsigned long long* status) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const int beg = pptr[k], end = pptr[k + 1];
        if (end < beg) {
            report(status, (int)k, kCodeInternal);
            continue;
        }
        for (int q = beg; q < end; ++q) {
            const int c = pidx[q];
            if (c != (int)k && !(c >= 0 && c < (int)k)) {
                report(status, (int)k, kCodeInternal);
                break;
            }
        }
    }
}

cudaError_t launch_verify_permuted(int n, const int* pptr, const int* pidx,
                                   unsigned long long* status, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    long long g = ((long long)n + 255) / 256;
    if (g > 65535) g = 65535;
    verify_permuted_k<<<(int)g, 256, 0, s>>>(n, pptr, pidx, status);
    return cudaGetLastError();
}

}  // namespace sptrsv
