// Internal interface between the C-ABI host code (api.cu) and the kernel
// translation units.  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace sptrsv {

// Everything a solve kernel needs.  The pattern is either the user's CSR or
// the plan's CSR of the transpose (then vmap maps entries to d_vals).
struct SolveParams {
    int n;
    const int* ptr;
    const int* idx;
    const int* vmap;      // nullptr: entry q has value vals[q]
    const void* vals;
    int diag_first;       // upper-triangular pattern: diagonal is a row's first entry
    int unit;
    const int* jlev;      // rows in level order
    const void* b;
    long long ldb;
    void* x;
    long long ldx;
    int nrhs;
    int* ticket;          // self-scheduled: next row group to hand out
    unsigned long long* status;
    SpinPolicy spin;
    int withhold;         // test hook: row whose result is never published (-1: none)
    const int* ipos;      // tiled solve in level order: position of each row in jlev
                          // (nullptr: tiles follow the substitution order)
    int kbeg, cnt;        // level-scheduled: this launch's slice of jlev
    void* xp;             // level-ordered solve: publication buffer in position
                          // order (nullptr: rows publish to x itself)
    const int* part_ptr;  // blocked solve: first position of each tile (nparts + 1
                          // entries; nullptr: tiles of tile_rows positions)
    int nparts;
    // FP64 accumulation of the published values (the FP32 solves of the
    // refined solve): xacc[i][c] = v (acc_first) or xacc[i][c] += v.
    // nullptr: off.  The copying forms then skip their store to x.
    double* xacc;
    long long ldacc;
    int acc_first;
    // the values are a pre-scaled copy (1/d(i) in the diagonal's slot, a_ij /
    // d(i) elsewhere; non-unit matrices): no division or scaling in the solve
    int prescaled;
};

// Adds (or stores) the published value v of row i, column c into p.xacc.
template <typename T>
__device__ __forceinline__ void accumulate_published(const SolveParams& p, long long i, int c,
                                                     T v) {
    double* a = p.xacc + i * p.ldacc + c;
    *a = p.acc_first ? (double)v : *a + (double)v;
}

// The value accumulate_with() will add to, loaded when the row is taken (off
// the dependency path) rather than after its publication, where the load
// would hold up the warp's other rows.
__device__ __forceinline__ double accumulate_base(const SolveParams& p, long long i, int c) {
    return (p.xacc && !p.acc_first) ? p.xacc[i * p.ldacc + c] : 0.0;
}
template <typename T>
__device__ __forceinline__ void accumulate_with(const SolveParams& p, long long i, int c, T v,
                                                double base) {
    p.xacc[i * p.ldacc + c] = p.acc_first ? (double)v : base + (double)v;
}

// Column structure of the column-wise solve (solve_column.cu): the CSR of
// the transpose of the system matrix, so row i lists the unknowns that
// depend on unknown i, plus the dependency counters.
struct ColumnParams {
    const int* ptr;
    const int* idx;
    const int* vmap;      // nullptr: entry q has value vals[q]
    int diag_first;       // the diagonal is a row's first entry (a lower system)
    int* count;           // working counters, reset from count0 before each solve
    const int* count0;    // off-diagonal entries of each row of the system
};

// ---- solve kernels (solve_self.cu, solve_level.cu, solve_mrhs.cu)
cudaError_t launch_prep_self(bool f64, int n, int nrhs, void* x, long long ldx, const void* b,
                             long long ldb, void* bcopy, int* ticket, int grid,
                             cudaStream_t s);
cudaError_t launch_self_k1(bool f64, int lanes, const SolveParams& p, int grid, int block,
                           cudaStream_t s);
cudaError_t launch_level_k1(bool f64, int lanes, const SolveParams& p, int block, cudaStream_t s);
cudaError_t launch_mrhs(bool f64, int lanes, bool self, const SolveParams& p, int grid, int block,
                        cudaStream_t s);
// Resident blocks per SM of the kernel a launch with these choices would use.
int self_blocks_per_sm(bool f64, int lanes, bool mrhs, bool map, int block);
// Tiled self-scheduled solve (solve_tiled.cu): tiles of `tile_rows`
// consecutive positions of the substitution order (p.ipos == nullptr) or of
// the level order jlev (p.ipos != nullptr); tile_rows * sizeof(T) <= 48 KB.
cudaError_t launch_tiled_k1(bool f64, int lanes, const SolveParams& p, int tile_rows, int grid,
                            int block, cudaStream_t s);
int tiled_blocks_per_sm(bool f64, int lanes, bool map, int block, int tile_rows);
// Chained self-scheduled solve (solve_chain.cu): tickets are segments of
// 32/lanes consecutive positions in substitution order, taken in the order
// `torder` (segment ids sorted by segment level); in-segment dependencies
// are forwarded between lanes by shuffle.
cudaError_t launch_chain_k1(bool f64, int lanes, const SolveParams& p, const int* torder,
                            int grid, int block, cudaStream_t s);
int chain_blocks_per_sm(bool f64, int lanes, bool map, int block);
// Column-wise self-scheduled solve (Alg. 4, solve_column.cu).  The prep
// launch sets x = b (unless x == b), count = count0 and the ticket to 0.
cudaError_t launch_column_counts(int n, const int* ptr, const int* idx, int* count,
                                 cudaStream_t s);
cudaError_t launch_prep_column(bool f64, const SolveParams& p, const ColumnParams& c, int grid,
                               cudaStream_t s);
cudaError_t launch_column_k1(bool f64, int lanes, const SolveParams& p, const ColumnParams& c,
                             int grid, int block, cudaStream_t s);
int column_blocks_per_sm(bool f64, int lanes, bool cmap, int block);
// Blocked self-scheduled solve on the level- or part-ordered copy
// (solve_blocked.cu): a block per tile of tile_rows consecutive positions,
// in-tile dependencies through shared memory (tile_rows * element size at
// most the device's opt-in shared memory per block, minus 128 B).
// cluster in {1, 2, 4, 8}: clusters of that many blocks take consecutive
// tiles together and read each other's tiles in distributed shared memory;
// grid must then be a multiple of cluster.
cudaError_t launch_blocked_k1(bool f64, int lanes, const SolveParams& p, int tile_rows, int grid,
                              int block, cudaStream_t s, int cluster = 1);
// Blocks of one launch that can be resident at once (0: the shape cannot run).
int blocked_resident_blocks(bool f64, int lanes, int cluster, int block, int tile_rows,
                            int num_sms);
// Resident blocks per SM of the level-ordered-copy form of self_solve_k1.
int self_perm_blocks_per_sm(bool f64, int lanes, int block);

// ---- partitioned solve (solve_parts.cu).  Positions t are in order of
// substitution (row t of a lower system, row n-1-t of an upper one).
// diff[0..n] (zeroed by the caller) gets +1 at f+1 and -1 at t+1 for every
// row at t whose farthest dependency is at f < t.
cudaError_t launch_part_spans(int n, const int* ptr, const int* idx, bool upper, int* diff,
                              cudaStream_t s);
// flag[t] = 1 where cover[t+1] (the exclusive scan of diff) is 0, or t = 0.
cudaError_t launch_block_flags(int n, const int* cover, int* flag, cudaStream_t s);
// start[scan[t]] = t where flag[t] (scan = exclusive scan of flag, n + 1
// entries); start[scan[n]] = n.
cudaError_t launch_flag_scatter(int n, const int* flag, const int* scan, int* start,
                                cudaStream_t s);
// depth[b] = max level of block b's rows (depth zeroed by the caller).
cudaError_t launch_block_depth(int n, bool upper, const int* lev, const int* bscan, int* depth,
                               cudaStream_t s);
// Part starts: balanced pieces of at most S rows of every block longer than
// S / 2, consecutive shorter blocks packed by windows of S / 2 positions.
cudaError_t launch_part_flags(int n, int S, const int* bscan, const int* bstart, int* flag,
                              cudaStream_t s);
cudaError_t launch_part_depth_keys(int np, int maxdepth, const int* pstart, const int* bscan,
                                   const int* depth, int* key, cudaStream_t s);
// piece[p] = index of part p among the parts of its block.
cudaError_t launch_part_piece(int np, const int* pstart, const int* bscan, const int* bstart,
                              const int* pscan, int* piece, cudaStream_t s);
// size[r] = rows of part horder[r]; *maxsize = max (zeroed by the caller).
// key[p] = slack of part p's block + piece[p] * levels per piece of the block.
cudaError_t launch_part_alap_keys(int np, int maxdepth, const int* pstart, const int* bscan,
                                  const int* bstart, const int* pscan, const int* depth,
                                  const int* piece, int* key, cudaStream_t s);
cudaError_t launch_part_sizes(int np, const int* horder, const int* pstart, int* size,
                              int* maxsize, cudaStream_t s);
// key[k] = prank[part of row jlev[k]].
cudaError_t launch_row_part_keys(int n, const int* jlev, bool upper, const int* pscan,
                                 const int* prank, int* key, cudaStream_t s);

// ---- level-ordered copy (permute.cu)
// lens[k] = length of row jlev[k].
cudaError_t launch_ordered_lengths(int n, const int* ptr, const int* jlev, int* lens,
                                   cudaStream_t s);
// Row k of the copy = row jlev[k] in fold order (rev: last entry first, for
// an upper row): pidx = ipos[idx] (skipped
// when pidx is nullptr, a values-only refresh), pvals = vals[vmap[q] or q];
// diag >= 0: pre-scaled by 1/d(i), with 1/d(i) in the diagonal's slot (the
// diagonal is the first entry of a row for diag = 1, the last for 0); -1:
// copied as they are (unit diagonal).
cudaError_t launch_permute_rows(bool f64, int n, const int* ptr, const int* idx, const int* vmap,
                                const void* vals, const int* jlev, const int* ipos,
                                const int* pptr, int* pidx, void* pvals, int grid,
                                cudaStream_t s, int diag, bool rev = false);
// Self-check: every entry of row k names k or an earlier position.
cudaError_t launch_verify_permuted(int n, const int* pptr, const int* pidx,
                                   unsigned long long* status, cudaStream_t s);

// ---- analysis kernels (analysis.cu)
cudaError_t launch_validate(int n, int nnz, const int* ptr, const int* idx, const void* vals,
                            bool f64, bool upper, bool unit, unsigned long long* status,
                            int grid, cudaStream_t s);
cudaError_t launch_level_sweep(int lanes, int n, const int* ptr, const int* idx, bool upper,
                               int* lev, int* ticket, int* nlev, unsigned long long* status,
                               SpinPolicy sp, int grid, int block, cudaStream_t s);
int level_sweep_blocks_per_sm(int lanes, int block);
// Levels of the graph of segments of 32/lanes consecutive positions in
// substitution order (chained solve); slev[] must start at -1, *ticket and
// *nslev at 0; *nslev ends as the number of segment levels.
cudaError_t launch_segment_sweep(int lanes, int n, const int* ptr, const int* idx, bool upper,
                                 int* slev, int* ticket, int* nslev, unsigned long long* status,
                                 SpinPolicy sp, int grid, int block, cudaStream_t s);
// Self-check: every out-of-segment dependency lies in a lower segment level
// (segments of R positions); failures are reported as internal.
cudaError_t launch_verify_segments(int n, int R, const int* ptr, const int* idx, bool upper,
                                   const int* slev, int nslev, unsigned long long* status,
                                   cudaStream_t s);
// count[keys[e]] += 1 for keys in [0, bins); any other key is reported as
// an internal error in *status and skipped.
cudaError_t launch_histogram(const int* keys, int m, int* count, int bins,
                             unsigned long long* status, cudaStream_t s);
// out[0..m]: exclusive prefix sums of in[0..m-1], out[m] = total.
cudaError_t launch_exclusive_scan(const int* in, int* out, int m, cudaStream_t s);
// Stable LSD radix sort of (keys, values = vals_in or the identity) by the
// low `bits` bits of the keys; sorted values land in vals_out.  Scratch:
// 4 int arrays of m entries and one of radix_hist_entries(m) entries (x2).
int radix_hist_entries(int m);
cudaError_t radix_sort_values(const int* keys_in, const int* vals_in, int m, int bits,
                              int* vals_out, int* k_a, int* v_a, int* k_b, int* v_b,
                              int* hist, int* hist_scan, unsigned long long* status,
                              cudaStream_t s);
cudaError_t launch_iota(int* out, int m, cudaStream_t s);
cudaError_t launch_row_of_entries(int n, const int* ptr, int* rowof, cudaStream_t s);
// out[e] = src[index[e]] for index in [0, src_len); others reported.
cudaError_t launch_gather(const int* src, int src_len, const int* index, int m, int* out,
                          unsigned long long* status, cudaStream_t s);
// ipos[perm[k]] = k (perm is a permutation of 0..n-1; checked before).
cudaError_t launch_inverse_perm(const int* perm, int n, int* ipos, cudaStream_t s);
// Self-check of level sets: every position of jlev holds a row of the
// level whose segment contains it, rows strictly increase inside a segment,
// ilev[0] = 0 and ilev[nlev] = n.  Failures are reported as internal.
cudaError_t launch_verify_levels(int n, int nlev, const int* lev, const int* ilev,
                                 const int* jlev, unsigned long long* status, cudaStream_t s);

// ---- Kahn's algorithm (kahn.cu, Sec. 4.4.1); dptr/didx: CSR of the
// transpose of the system (the outgoing edges of every row)
cudaError_t launch_kahn_roots(int n, const int* count0, int* count, int* lev, int* queue,
                              int* qend, cudaStream_t s);
cudaError_t launch_kahn_level(const int* dptr, const int* didx, int* count, int* lev, int* queue,
                              int* qend, int n, int first, int last, int level,
                              unsigned long long* status, int max_grid, cudaStream_t s);
int kahn_persistent_blocks_per_sm(int block);
// cnt[0] = roots queued by launch_kahn_roots, cnt[1] = cnt[2] = 0; on exit
// cnt[3] = rows leveled and *nlev_out = levels.  ctl: 3 ints of scratch.
// Levels of at most `narrow` rows run on block 0 alone.  With probe_level
// > 0, the launch gives up (*nlev_out = -1) when fewer than
// level * probe_min_avg rows are leveled after probe_level levels, unless
// the levels are still widening, in which case it looks again (once) at
// four times that level with a 1.5 times larger average.
cudaError_t launch_kahn_persistent(const int* dptr, const int* didx, int* count, int* lev,
                                   int* queue, int* cnt, int* ctl, int n, int narrow,
                                   int probe_level, int probe_min_avg,
                                   unsigned long long* arrivals, int* nlev_out,
                                   unsigned long long* status, long long limit, int grid,
                                   int block, cudaStream_t s);

// ---- refinement in one pass (refine.cu): on the level-ordered copy, K + 1
// steps m = 0..K per row (residual in FP64, correction in FP32, update in
// FP64), published per step in position order.
constexpr int kRefineMaxSteps = 4;  // K <= kRefineMaxSteps per pass
struct RefineParams {
    int n;
    const int* ptr;        // level-ordered copy: position k holds row jlev[k]
    const int* idx;        // columns renumbered to positions
    const double* v64;     // FP64 values of the copy (pre-scaled by 1/d(i) unless unit)
    const float* v32;      // FP32 values of the copy (pre-scaled likewise)
    const int* jlev;
    int unit, diag_first;
    const double* b;
    long long ldb;
    double* x;             // in: initial guess (has_init); out: x^{K+1}
    long long ldx;
    int has_init;
    int K;
    float* dpub;           // [K+1][n] corrections d^m, position order
    double* xpub;          // [K+1][n] iterates x^m, position order
    int* ticket;
    unsigned long long* status;
    unsigned long long* rmax;  // [K+1] max |r^m| (bits of a non-negative double)
    unsigned long long* xmax;  // [K+1] max |x^m|
    SpinPolicy spin;
};
cudaError_t launch_refine_pass(int lanes, const RefineParams& r, int grid, int block,
                               cudaStream_t s);
int refine_blocks_per_sm(int lanes, int block);

// ---- auxiliary kernels (aux.cu)
cudaError_t launch_grad_vals(bool f64, int lanes, int n, const int* ptr, const int* idx, bool unit,
                             const void* y, long long ldy, const void* x, long long ldx, int k,
                             void* g, cudaStream_t s, int grid);
// r = b - A x in FP64; writes r (nullable, [n][ldr]) and r32 (nullable,
// contiguous [n][k]); stats (nullable): atomicMax of max|r| into stats[0],
// of max|x| into stats[2] and, if want_norm, of max_i sum_j |A_ij| into
// stats[1].
cudaError_t launch_residual(int n, long long nnz, const int* ptr, const int* idx,
                            const double* vals, bool unit, int k, const double* b, long long ldb,
                            const double* x, long long ldx, double* r, long long ldr, float* r32,
                            unsigned long long* stats, bool want_norm, int grid, cudaStream_t s);
// x = d (first) or x += d, FP64 x [n][ldx], FP32 d contiguous [n][k];
// atomicMax of max|x| into *xmax.
cudaError_t launch_update(int n, int k, double* x, long long ldx, const float* d, bool first,
                          unsigned long long* xmax, int grid, cudaStream_t s);
// out32 = (float) in64 over [n][k] (in strided by ldin, out contiguous);
// atomicMax of max|in| into *amax (nullable).
cudaError_t launch_to_f32(int n, int k, const double* in, long long ldin, float* out,
                          unsigned long long* amax, int grid, cudaStream_t s);

}  // namespace sptrsv
