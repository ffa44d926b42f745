// C ABI of the solver (declared in include/sptrsv.h): argument checking,
// plan ownership, the setup sequence of Sec. 4.4 and the launch sequences of
// the solves.  All arithmetic runs in the kernels of the other files.
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "internal.h"
#include "sptrsv.h"

using namespace sptrsv;

namespace {

thread_local int g_last_error_row = -1;
thread_local char g_last_cuda[256] = "";

sptrsv_status_t cuda_fail(cudaError_t e) {
    snprintf(g_last_cuda, sizeof(g_last_cuda), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SPTRSV_ERR_OOM : SPTRSV_ERR_CUDA;
}

#define CK(expr)                                   \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) return cuda_fail(_e); \
    } while (0)

#define ST(expr)                                \
    do {                                        \
        sptrsv_status_t _s = (expr);            \
        if (_s != SPTRSV_OK) return _s;         \
    } while (0)

struct Levels {
    int nlev = 0;
    int* lev = nullptr;
    int* ilev = nullptr;
    int* jlev = nullptr;
    int* ipos = nullptr;  // inverse of jlev (level-order tiles)
    std::vector<int> h_ilev;
    // Chained solve, per log2(lanes): segment ids in segment-level order
    // (built on first use) and the number of segment levels.
    int* torder[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    int nslev[6] = {0, 0, 0, 0, 0, 0};
    // Level-ordered copy (SPTRSV_ALGO_SELF_PERMUTED, built on first use):
    // row k = row jlev[k], columns renumbered to positions, values copied;
    // xp is the position-ordered publication buffer of its solves.
    int* pptr = nullptr;
    int* pidx = nullptr;
    void* pvals = nullptr;
    void* xp = nullptr;
    // Column-wise solve (SPTRSV_ALGO_SELF_COLUMN, built on first use): the
    // dependency count of every row and the working counters.
    int* count0 = nullptr;
    int* count = nullptr;
    int method = SPTRSV_ANALYSIS_SWEEP;  // the analysis that produced these levels
    // Part-ordered copy (SPTRSV_ALGO_SELF_PARTITIONED, built on first use and
    // again when the part size changes): position k holds row qord[k], rows
    // in parts of qS consecutive rows, by level inside a part; columns
    // renumbered to positions (qipos); xq is the publication buffer of its
    // solves (position order).
    // qpart: first position of each part (qnparts + 1 entries, parts in the
    // order they are handed out), qmaxpart the longest part, qnblocks the
    // independent blocks the substitution order splits into.
    int qS = 0;
    int* qord = nullptr;
    int* qipos = nullptr;
    int* qptr = nullptr;
    int* qidx = nullptr;
    void* qvals = nullptr;
    void* xq = nullptr;
    int* qpart = nullptr;
    int qnparts = 0, qmaxpart = 0, qnblocks = 0;
    // FP32 values and publication buffers of the level- and part-ordered
    // copies of an F64 plan, for the FP32 solves of the refined solve (built
    // on first use from the plan's FP32 copy of the values).
    void* pvals32 = nullptr;
    void* xp32 = nullptr;
    void* qvals32 = nullptr;
    void* xq32 = nullptr;
    // multi-RHS solves on the level-ordered copy: publication buffer
    // [n][nrhs] in position order (grown on demand)
    void* xpm = nullptr;
    size_t xpm_bytes = 0;
};

void free_parts(Levels& L) {
    cudaFree(L.qord);
    cudaFree(L.qipos);
    cudaFree(L.qptr);
    cudaFree(L.qidx);
    cudaFree(L.qvals);
    cudaFree(L.xq);
    cudaFree(L.qpart);
    cudaFree(L.qvals32);
    cudaFree(L.xq32);
    L.qord = L.qipos = L.qptr = L.qidx = L.qpart = nullptr;
    L.qvals = L.xq = L.qvals32 = L.xq32 = nullptr;
    L.qS = L.qnparts = L.qmaxpart = L.qnblocks = 0;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int pow2_at_least(double v) {
    int w = 1;
    while (w < v && w < 32) w <<= 1;
    return w;
}

// Default sub-warp width: enough lanes for the average number of
// off-diagonal entries of a row, at least 2, at most 32.
int default_lanes(int n, int nnz) {
    if (n <= 0) return 4;
    const double off = (double)nnz / n - 1.0;
    int w = pow2_at_least(off);
    return w < 2 ? 2 : w;
}

// Default sub-warp width of the multi-RHS kernels: one lane per column up to
// 16 lanes, beyond that several columns per lane.  A narrower group holds
// more rows per warp, so more rows wait ahead of the dependency frontier
// (128^3 L factor, k = 32: 1.24 ms with 16 lanes against 1.98 ms with 32).
int mrhs_lanes(int nrhs) {
    int w = pow2_at_least(nrhs);
    if (w < 4) w = 4;
    return w > 16 ? 16 : w;
}

bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &st) != cudaSuccess) return false;
    return st != cudaStreamCaptureStatusNone;
}

int bits_for(int max_key) {
    int b = 0;
    while (b < 31 && (max_key >> b) != 0) ++b;
    return b;
}

long long env_ll(const char* name, long long dflt) {
    const char* v = getenv(name);
    if (!v || !*v) return dflt;
    char* end = nullptr;
    long long x = strtoll(v, &end, 0);
    return (end && *end == 0 && x > 0) ? x : dflt;
}

}  // namespace

struct sptrsv_plan_s {
    int device = 0;
    int num_sms = 1;
    int n = 0, nnz = 0;
    bool f64 = true, upper = false, unit = false;
    const int* rowptr = nullptr;
    const int* colidx = nullptr;
    const void* vals = nullptr;
    Levels fwd, trn;
    bool has_trans = false;     // transposed pattern and its levels
    bool has_tpattern = false;  // transposed pattern
    int* tptr = nullptr;
    int* tidx = nullptr;
    int* tmap = nullptr;
    int* counters = nullptr;  // [0] ticket, [1] level count
    unsigned long long* status = nullptr;
    void* bcopy = nullptr;
    size_t bcopy_bytes = 0;
    float* vals32 = nullptr;
    float* r32 = nullptr;
    float* d32 = nullptr;
    size_t rd_elems = 0;
    unsigned long long* stats = nullptr;  // [0] max|r| [1] |A|_inf [2] max|x| [3] max|b|
    // one-pass refinement (refine.cu): step buffers and per-step norms
    void* rf_dpub = nullptr;
    void* rf_xpub = nullptr;
    size_t rf_bytes = 0;
    unsigned long long* rf_norms = nullptr;  // [0, S) max|r^m|, [S, 2S) max|x^m|
    double anorm = -1.0;                     // ||A||_inf of the current values (-1: unknown)
    int lanes = 4, block = 256, max_blocks = 0;
    // per-algorithm single-RHS shapes (lanes 0: use the plan's shape)
    int alg_lanes[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int alg_block[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int alg_max_blocks[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // multi-RHS launch shape: width (0: chosen from nrhs), block (0: the
    // single-RHS one), grid cap (-1: the single-RHS one)
    int mrhs_lanes = 0, mrhs_block = 0, mrhs_max_blocks = -1;
    int tile_rows = 2048;
    bool tile_level_order = false;
    int part_rows = 0;   // partitioned solve: rows per part (0: automatic)
    int part_cluster = 1;  // partitioned solve: blocks per thread-block cluster
    sptrsv_algo_t default_algo = SPTRSV_ALGO_SELF;  // SPTRSV_ALGO_AUTO and refined solves
    sptrsv_refine_t refine_mode = SPTRSV_REFINE_STAGED;
    int smem_optin = 0;  // shared memory a block may opt in to
    SpinPolicy spin{1ll << 24, 256, 128};
    int withhold = -1;
    double analysis_ms = 0.0;
    bool prof = false;
    std::vector<cudaEvent_t> ev;  // start/stop pairs
    size_t ev_used = 0;
    int last_launches = 0;
};

namespace {

void free_levels(Levels& L) {
    cudaFree(L.lev);
    cudaFree(L.ilev);
    cudaFree(L.jlev);
    cudaFree(L.ipos);
    for (int* t : L.torder) cudaFree(t);
    cudaFree(L.pptr);
    cudaFree(L.pidx);
    cudaFree(L.pvals);
    cudaFree(L.xp);
    cudaFree(L.pvals32);
    cudaFree(L.xp32);
    cudaFree(L.xpm);
    cudaFree(L.count0);
    cudaFree(L.count);
    free_parts(L);
    L = Levels();
}

void destroy(sptrsv_plan_t P) {
    if (!P) return;
    DeviceGuard g(P->device);
    free_levels(P->fwd);
    free_levels(P->trn);
    cudaFree(P->tptr);
    cudaFree(P->tidx);
    cudaFree(P->tmap);
    cudaFree(P->counters);
    cudaFree(P->status);
    cudaFree(P->bcopy);
    cudaFree(P->vals32);
    cudaFree(P->r32);
    cudaFree(P->d32);
    cudaFree(P->stats);
    cudaFree(P->rf_dpub);
    cudaFree(P->rf_xpub);
    cudaFree(P->rf_norms);
    for (cudaEvent_t e : P->ev) cudaEventDestroy(e);
    delete P;
}

// Reads and clears the status word (synchronises s).  Returns the code and
// stores the row.
sptrsv_status_t take_status(sptrsv_plan_t P, cudaStream_t s, int* row) {
    unsigned long long h = kStatusClear;
    CK(cudaMemcpyAsync(&h, P->status, sizeof(h), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (row) *row = -1;
    if (h == kStatusClear) return SPTRSV_OK;
    CK(cudaMemsetAsync(P->status, 0xff, sizeof(unsigned long long), s));
    CK(cudaStreamSynchronize(s));
    if (row) *row = (int)(h >> 32);
    return (sptrsv_status_t)(unsigned)(h & 0xffffffffu);
}

sptrsv_status_t sweep_levels(sptrsv_plan_t P, const int* ptr, const int* idx, bool upper,
                             Levels& L, int* nlev_out, cudaStream_t s);
sptrsv_status_t level_sets(sptrsv_plan_t P, Levels& L, int nlev, cudaStream_t s);

// Levels by Kahn's algorithm (Sec. 4.4.1): dptr/didx is the CSR of the
// transpose of the system (row i lists the rows that depend on i).  The
// host-loop form launches once per level and reads the queue end back after
// each launch; the persistent form runs every level in one cooperative
// launch.  Writes L.lev (allocated by the caller) and *nlev; synchronises s.
sptrsv_status_t kahn_levels(sptrsv_plan_t P, const int* ptr, const int* idx, const int* dptr,
                            const int* didx, bool persistent, bool probe, Levels& L, int* nlev,
                            cudaStream_t s) {
    const int n = P->n;
    int* scratch = nullptr;
    // Layout (ints): [0, 2) the 64-bit barrier counter, which must be 8-byte
    // aligned and so comes first (cudaMalloc returns 256-byte aligned
    // memory); [2, 6) the queue end / rotating level counters (the roots are
    // counted in [2]; [5] = rows leveled by the persistent form); [6] level
    // count; [7, 10) the persistent form's narrow-run state; [10, 12) pad;
    // then count0, count, queue.
    CK(cudaMalloc(&scratch, sizeof(int) * (3 * (size_t)n + 12)));
    unsigned long long* arrivals = (unsigned long long*)scratch;
    int* qend = scratch + 2;
    int* nlev_dev = scratch + 6;
    int* ctl = scratch + 7;
    int* count0 = scratch + 12;
    int* count = count0 + n;
    int* queue = count + n;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 12 * sizeof(int), s);
    if (e == cudaSuccess) e = launch_column_counts(n, ptr, idx, count0, s);
    if (e == cudaSuccess) e = launch_kahn_roots(n, count0, count, L.lev, queue, qend, s);
    int h_last = 0, level = 0;
    if (e == cudaSuccess && persistent) {
        // One block of 1024 threads per SM keeps the grid barrier short (one
        // arrival per SM); a level with at most one row per warp of a block
        // runs on block 0 alone.
        int block = (int)env_ll("SPTRSV_KAHN_BLOCK", 1024);
        if (block < 64 || block > 1024 || block % 32 != 0) block = 1024;
        long long per_sm = env_ll("SPTRSV_KAHN_BLOCKS_PER_SM", 1);
        const long long fit = kahn_persistent_blocks_per_sm(block);
        if (per_sm > fit) per_sm = fit;
        long long grid = per_sm * P->num_sms;
        if (grid < 1) grid = 1;
        const int narrow = (int)env_ll("SPTRSV_KAHN_NARROW", block / 32);
        // Probe (automatic method only): after 256 levels, fewer than 112
        // rows per level on average means a deep, narrow graph, where a
        // grid barrier per level loses to the sweep (measured: 2.2-3.6 us
        // per level against the sweep's 1.2-1.3 us on such graphs); levels
        // still widening at that point are judged again at level 1024.
        const int probe_level = probe ? 256 : 0;
        e = launch_kahn_persistent(dptr, didx, count, L.lev, queue, qend, ctl, n, narrow,
                                   probe_level, 112, arrivals, nlev_dev, P->status,
                                   P->spin.limit, (int)grid, block, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&level, nlev_dev, sizeof(int),
                                                  cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_last, qend + 3, sizeof(int),
                                                  cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    } else if (e == cudaSuccess) {
        // the paper's driver: one launch and one copy of the queue end per level
        e = cudaMemcpyAsync(&h_last, qend, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        int first = 0;
        while (e == cudaSuccess && h_last > first) {
            e = launch_kahn_level(dptr, didx, count, L.lev, queue, qend, n, first, h_last, level,
                                  P->status, P->num_sms * 16, s);
            int nl = h_last;
            if (e == cudaSuccess) e = cudaMemcpyAsync(&nl, qend, sizeof(int),
                                                      cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            first = h_last;
            h_last = nl;
            ++level;
        }
    }
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    int row = -1;
    ST(take_status(P, s, &row));
    if (probe && level == -1) {  // gave up early: the caller runs the sweep
        *nlev = -1;
        return SPTRSV_OK;
    }
    if (h_last != n || level < 1) return SPTRSV_ERR_INTERNAL;  // every row must be leveled
    *nlev = level;
    return SPTRSV_OK;
}

// Level analysis of one pattern (Sec. 4.1): the levels (sync-free sweep, or
// Kahn's algorithm given the dependents' structure dptr/didx), then the
// bucket sort into level sets.  Synchronises s.
sptrsv_status_t build_levels(sptrsv_plan_t P, const int* ptr, const int* idx, bool upper,
                             Levels& L, cudaStream_t s, int method = SPTRSV_ANALYSIS_AUTO,
                             const int* dptr = nullptr, const int* didx = nullptr) {
    const int n = P->n;
    CK(cudaMalloc(&L.lev, sizeof(int) * (size_t)n));
    CK(cudaMemsetAsync(L.lev, 0xff, sizeof(int) * (size_t)n, s));
    CK(cudaMemsetAsync(P->counters, 0, 2 * sizeof(int), s));
    int nlev = -1;
    const bool kahn = method == SPTRSV_ANALYSIS_KAHN_HOST_LOOP ||
                      method == SPTRSV_ANALYSIS_KAHN_PERSISTENT ||
                      (method == SPTRSV_ANALYSIS_AUTO && dptr);
    L.method = SPTRSV_ANALYSIS_SWEEP;
    if (kahn) {
        ST(kahn_levels(P, ptr, idx, dptr, didx, method != SPTRSV_ANALYSIS_KAHN_HOST_LOOP,
                       method == SPTRSV_ANALYSIS_AUTO, L, &nlev, s));
        if (nlev >= 0)
            L.method = method == SPTRSV_ANALYSIS_KAHN_HOST_LOOP ? SPTRSV_ANALYSIS_KAHN_HOST_LOOP
                                                                : SPTRSV_ANALYSIS_KAHN_PERSISTENT;
    }
    if (nlev < 0) {  // the sweep, by choice or after Kahn gave up
        if (kahn) {
            CK(cudaMemsetAsync(L.lev, 0xff, sizeof(int) * (size_t)n, s));
            CK(cudaMemsetAsync(P->counters, 0, 2 * sizeof(int), s));
        }
        ST(sweep_levels(P, ptr, idx, upper, L, &nlev, s));
    }
    return level_sets(P, L, nlev, s);
}

// Levels by the sync-free sweep (analysis.cu).  Writes L.lev and *nlev;
// synchronises s.
sptrsv_status_t sweep_levels(sptrsv_plan_t P, const int* ptr, const int* idx, bool upper,
                             Levels& L, int* nlev_out, cudaStream_t s) {
    const int n = P->n;
    // One lane per ~4 entries of an average row (a chunk), so short rows get a
    // lane each and a ticket holds many consecutive rows; a moderate grid
    // keeps the polling traffic down.
    int lanes = (int)env_ll("SPTRSV_SWEEP_LANES", 0);
    if (!(lanes == 1 || lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32))
        lanes = pow2_at_least(((double)P->nnz / (n > 0 ? n : 1) - 1.0) / kChunk);
    const int block = 256;
    const int R = 32 / lanes;
    const long long tickets = ((long long)n + R - 1) / R;
    const long long want_blocks = (tickets + block / 32 - 1) / (block / 32);
    long long per_sm = env_ll("SPTRSV_SWEEP_BLOCKS_PER_SM", 4);
    const long long fit = level_sweep_blocks_per_sm(lanes, block);
    if (per_sm > fit) per_sm = fit;
    long long grid = per_sm * P->num_sms;
    if (grid > want_blocks) grid = want_blocks;
    if (grid < 1) grid = 1;
    CK(launch_level_sweep(lanes, n, ptr, idx, upper, L.lev, P->counters, P->counters + 1,
                          P->status, P->spin, (int)grid, block, s));
    int nlev = 0;
    CK(cudaMemcpyAsync(&nlev, P->counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    int row = -1;
    ST(take_status(P, s, &row));  // synchronises
    *nlev_out = nlev;
    return SPTRSV_OK;
}

// Level sets from L.lev (Sec. 4.1): histogram, exclusive scan to ilev, a
// stable radix sort of the rows by level to jlev (ascending rows inside a
// level), a self-check, and the inverse permutation ipos.  Synchronises s.
sptrsv_status_t level_sets(sptrsv_plan_t P, Levels& L, int nlev, cudaStream_t s) {
    const int n = P->n;
    int row = -1;
    L.nlev = nlev;
    CK(cudaMalloc(&L.ilev, sizeof(int) * (size_t)(nlev + 1)));
    CK(cudaMalloc(&L.jlev, sizeof(int) * (size_t)n));
    CK(cudaMalloc(&L.ipos, sizeof(int) * (size_t)n));
    int* count = nullptr;
    int* scratch = nullptr;
    const int hist_n = radix_hist_entries(n);
    const size_t scratch_ints = (size_t)nlev + 4 * (size_t)n + 2 * (size_t)hist_n;
    CK(cudaMalloc(&scratch, sizeof(int) * scratch_ints));
    count = scratch;
    int* k_a = count + nlev;
    int* v_a = k_a + n;
    int* k_b = v_a + n;
    int* v_b = k_b + n;
    int* hist = v_b + n;
    int* hist_scan = hist + hist_n;
    sptrsv_status_t rc = SPTRSV_OK;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)nlev, s);
    if (e == cudaSuccess) e = launch_histogram(L.lev, n, count, nlev, P->status, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(count, L.ilev, nlev, s);
    if (e == cudaSuccess)
        e = radix_sort_values(L.lev, nullptr, n, bits_for(nlev - 1), L.jlev, k_a, v_a, k_b, v_b,
                              hist, hist_scan, P->status, s);
    if (e == cudaSuccess) e = launch_verify_levels(n, nlev, L.lev, L.ilev, L.jlev, P->status, s);
    if (e == cudaSuccess) {
        L.h_ilev.resize((size_t)nlev + 1);
        e = cudaMemcpyAsync(L.h_ilev.data(), L.ilev, sizeof(int) * (size_t)(nlev + 1),
                            cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e);
    cudaFree(scratch);
    if (rc == SPTRSV_OK) rc = take_status(P, s, &row);
    // jlev is now known to be a permutation: invert it for level-order tiles.
    if (rc == SPTRSV_OK) {
        e = launch_inverse_perm(L.jlev, n, L.ipos, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    return rc;
}

// CSR of A^T (the CSC of A, Sec. 3.2) with a value map, and its levels.
sptrsv_status_t build_transpose_pattern(sptrsv_plan_t P, cudaStream_t s);
sptrsv_status_t build_transpose(sptrsv_plan_t P, cudaStream_t s) {
    if (P->has_trans) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    ST(build_transpose_pattern(P, s));
    ST(build_levels(P, P->tptr, P->tidx, !P->upper, P->trn, s, SPTRSV_ANALYSIS_AUTO, P->rowptr,
                    P->colidx));
    P->has_trans = true;
    return SPTRSV_OK;
}

// The transposed pattern alone (no levels), built once.
sptrsv_status_t build_transpose_pattern(sptrsv_plan_t P, cudaStream_t s) {
    if (P->has_tpattern) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    const int n = P->n, nnz = P->nnz;
    cudaFree(P->tptr);  // left over from a failed attempt, if any
    cudaFree(P->tidx);
    cudaFree(P->tmap);
    P->tptr = P->tidx = P->tmap = nullptr;
    CK(cudaMalloc(&P->tptr, sizeof(int) * (size_t)(n + 1)));
    CK(cudaMalloc(&P->tidx, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1)));
    CK(cudaMalloc(&P->tmap, sizeof(int) * (size_t)(nnz > 0 ? nnz : 1)));
    const int hist_n = radix_hist_entries(nnz);
    const size_t scratch_ints = (size_t)n + 5 * (size_t)nnz + 2 * (size_t)hist_n;
    int* scratch = nullptr;
    CK(cudaMalloc(&scratch, sizeof(int) * scratch_ints));
    int* count = scratch;
    int* k_a = count + n;
    int* v_a = k_a + nnz;
    int* k_b = v_a + nnz;
    int* v_b = k_b + nnz;
    int* rowof = v_b + nnz;
    int* hist = rowof + nnz;
    int* hist_scan = hist + hist_n;
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)n, s);
    if (e == cudaSuccess) e = launch_histogram(P->colidx, nnz, count, n, P->status, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(count, P->tptr, n, s);
    if (e == cudaSuccess)
        e = radix_sort_values(P->colidx, nullptr, nnz, bits_for(n - 1), P->tmap, k_a, v_a, k_b,
                              v_b, hist, hist_scan, P->status, s);
    if (e == cudaSuccess) e = launch_row_of_entries(n, P->rowptr, rowof, s);
    if (e == cudaSuccess) e = launch_gather(rowof, nnz, P->tmap, nnz, P->tidx, P->status, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(scratch);
    if (e != cudaSuccess) return cuda_fail(e);
    int row = -1;
    sptrsv_status_t rc = take_status(P, s, &row);
    // The transposed pattern must itself be a valid triangle of the other
    // kind (a self-check: any failure here is a library bug).
    if (rc == SPTRSV_OK) {
        CK(launch_validate(n, nnz, P->tptr, P->tidx, nullptr, P->f64, !P->upper, true, P->status,
                           P->num_sms * 32, s));
        rc = take_status(P, s, &row);
    }
    if (rc != SPTRSV_OK) return SPTRSV_ERR_INTERNAL;
    P->has_tpattern = true;
    return SPTRSV_OK;
}

int log2_lanes(int lanes) {
    int k = 0;
    while ((1 << k) < lanes) ++k;
    return k;
}

// Ticket order of the chained solve for one direction and sub-warp width:
// segments of R = 32/lanes consecutive positions of the substitution order,
// their levels in the segment graph (a sweep like the row levels of
// Sec. 4.1), and the segment ids stably sorted by that level.  Built once
// per (direction, lanes); allocates and synchronises s.
sptrsv_status_t build_chain(sptrsv_plan_t P, bool trans, int lanes, cudaStream_t s) {
    Levels& L = trans ? P->trn : P->fwd;
    const int k = log2_lanes(lanes);
    if (L.torder[k]) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    const int n = P->n;
    const int R = 32 / lanes;
    const int nseg = (int)(((long long)n + R - 1) / R);
    const int* ptr = trans ? P->tptr : P->rowptr;
    const int* idx = trans ? P->tidx : P->colidx;
    const bool upper = trans ? !P->upper : P->upper;
    const int hist_n = radix_hist_entries(nseg);
    int* scratch = nullptr;
    CK(cudaMalloc(&scratch, sizeof(int) * (5 * (size_t)nseg + 2 * (size_t)hist_n)));
    int* slev = scratch;
    int* k_a = slev + nseg;
    int* v_a = k_a + nseg;
    int* k_b = v_a + nseg;
    int* v_b = k_b + nseg;
    int* hist = v_b + nseg;
    int* hist_scan = hist + hist_n;
    int* torder = nullptr;
    cudaError_t e = cudaMalloc(&torder, sizeof(int) * (size_t)nseg);
    if (e != cudaSuccess) {
        cudaFree(scratch);
        return cuda_fail(e);
    }
    const int block = 256;
    const long long want_blocks = ((long long)nseg + block / 32 - 1) / (block / 32);
    long long grid = env_ll("SPTRSV_SWEEP_BLOCKS_PER_SM", 4) * P->num_sms;
    if (grid > want_blocks) grid = want_blocks;
    if (grid < 1) grid = 1;
    int nslev = 0;
    e = cudaMemsetAsync(slev, 0xff, sizeof(int) * (size_t)nseg, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->counters, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess)
        e = launch_segment_sweep(lanes, n, ptr, idx, upper, slev, P->counters, P->counters + 1,
                                 P->status, P->spin, (int)grid, block, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nslev, P->counters + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    sptrsv_status_t rc = e == cudaSuccess ? SPTRSV_OK : cuda_fail(e);
    int row = -1;
    if (rc == SPTRSV_OK) rc = take_status(P, s, &row);
    if (rc == SPTRSV_OK && (nslev < 1 || nslev > nseg)) rc = SPTRSV_ERR_INTERNAL;
    if (rc == SPTRSV_OK) {
        e = radix_sort_values(slev, nullptr, nseg, bits_for(nslev - 1), torder, k_a, v_a, k_b,
                              v_b, hist, hist_scan, P->status, s);
        if (e == cudaSuccess)
            e = launch_verify_segments(n, R, ptr, idx, upper, slev, nslev, P->status, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(e);
        if (rc == SPTRSV_OK && take_status(P, s, &row) != SPTRSV_OK) rc = SPTRSV_ERR_INTERNAL;
    }
    cudaFree(scratch);
    if (rc != SPTRSV_OK) {
        if (row >= 0) g_last_error_row = row;
        cudaFree(torder);
        return rc;
    }
    L.torder[k] = torder;
    L.nslev[k] = nslev;
    return SPTRSV_OK;
}

// How the copies store a row's values: pre-scaled by 1/d(i) with the
// diagonal's slot at the row's start (1) or end (0) for a non-unit matrix,
// as they are (-1) for a unit one.
int copy_diag(sptrsv_plan_t P, bool trans) {
    if (P->unit) return -1;
    return (trans ? !P->upper : P->upper) ? 1 : 0;
}

// Level-ordered copy of one direction's pattern and values (Sec. 4.3,
// remark 2: preordering by level), its self-check and the publication
// buffer.  Built once per direction; allocates and synchronises s.
sptrsv_status_t build_permuted(sptrsv_plan_t P, bool trans, cudaStream_t s) {
    Levels& L = trans ? P->trn : P->fwd;
    if (L.pptr) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    const int n = P->n, nnz = P->nnz;
    const size_t esize = P->f64 ? sizeof(double) : sizeof(float);
    const int* ptr = trans ? P->tptr : P->rowptr;
    const int* idx = trans ? P->tidx : P->colidx;
    const int* vmap = trans ? P->tmap : nullptr;
    int *pptr = nullptr, *pidx = nullptr, *lens = nullptr;
    void *pvals = nullptr, *xp = nullptr;
    cudaError_t e = cudaMalloc(&pptr, sizeof(int) * ((size_t)n + 1));
    if (e == cudaSuccess) e = cudaMalloc(&pidx, sizeof(int) * (nnz > 0 ? (size_t)nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&pvals, esize * (nnz > 0 ? (size_t)nnz : 1));
    if (e == cudaSuccess) e = cudaMalloc(&xp, esize * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&lens, sizeof(int) * (size_t)n);
    if (e == cudaSuccess) e = launch_ordered_lengths(n, ptr, L.jlev, lens, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(lens, pptr, n, s);
    if (e == cudaSuccess)
        e = launch_permute_rows(P->f64, n, ptr, idx, vmap, P->vals, L.jlev, L.ipos, pptr, pidx,
                                pvals, P->num_sms * 16, s, copy_diag(P, trans),
                                trans ? !P->upper : P->upper);
    if (e == cudaSuccess) e = launch_verify_permuted(n, pptr, pidx, P->status, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    sptrsv_status_t rc = e == cudaSuccess ? SPTRSV_OK : cuda_fail(e);
    int row = -1;
    if (rc == SPTRSV_OK && take_status(P, s, &row) != SPTRSV_OK) rc = SPTRSV_ERR_INTERNAL;
    cudaFree(lens);
    if (rc != SPTRSV_OK) {
        cudaFree(pptr);
        cudaFree(pidx);
        cudaFree(pvals);
        cudaFree(xp);
        return rc;
    }
    L.pptr = pptr;
    L.pidx = pidx;
    L.pvals = pvals;
    L.xp = xp;
    return SPTRSV_OK;
}

// Dependency counters of the column-wise solve (Alg. 4) for one direction:
// count0[r] = off-diagonal entries of row r of the system matrix.  The
// column structure is the CSR of the system's transpose, so the forward
// solve needs the transposed pattern too.  Allocates and synchronises s.
sptrsv_status_t build_column(sptrsv_plan_t P, bool trans, cudaStream_t s) {
    Levels& L = trans ? P->trn : P->fwd;
    if (L.count0) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    ST(build_transpose(P, s));
    int *count0 = nullptr, *count = nullptr;
    cudaError_t e = cudaMalloc(&count0, sizeof(int) * (size_t)P->n);
    if (e == cudaSuccess) e = cudaMalloc(&count, sizeof(int) * (size_t)P->n);
    if (e == cudaSuccess)
        e = launch_column_counts(P->n, trans ? P->tptr : P->rowptr, trans ? P->tidx : P->colidx,
                                 count0, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(count0);
        cudaFree(count);
        return cuda_fail(e);
    }
    L.count0 = count0;
    L.count = count;
    return SPTRSV_OK;
}

// Re-gathers the values of every level-ordered copy from the plan's values.
cudaError_t refresh_permuted(sptrsv_plan_t P, cudaStream_t s) {
    for (int d = 0; d < 2; ++d) {
        Levels& L = d ? P->trn : P->fwd;
        if (!L.pvals) continue;
        cudaError_t e = launch_permute_rows(P->f64, P->n, d ? P->tptr : P->rowptr,
                                            d ? P->tidx : P->colidx, d ? P->tmap : nullptr,
                                            P->vals, L.jlev, L.ipos, L.pptr, nullptr, L.pvals,
                                            P->num_sms * 16, s, copy_diag(P, d),
                                            d ? !P->upper : P->upper);
        if (e != cudaSuccess) return e;
    }
    for (int d = 0; d < 2; ++d) {
        Levels& L = d ? P->trn : P->fwd;
        if (!L.qvals) continue;
        cudaError_t e = launch_permute_rows(P->f64, P->n, d ? P->tptr : P->rowptr,
                                            d ? P->tidx : P->colidx, d ? P->tmap : nullptr,
                                            P->vals, L.qord, L.qipos, L.qptr, nullptr, L.qvals,
                                            P->num_sms * 16, s, copy_diag(P, d),
                                            d ? !P->upper : P->upper);
        if (e != cudaSuccess) return e;
    }
    // the FP32 copies of the refined solve, from the refreshed FP32 values
    for (int d = 0; d < 2 && P->vals32; ++d) {
        Levels& L = d ? P->trn : P->fwd;
        for (int parts = 0; parts < 2; ++parts) {
            void* v = parts ? L.qvals32 : L.pvals32;
            if (!v) continue;
            cudaError_t e = launch_permute_rows(
                false, P->n, d ? P->tptr : P->rowptr, d ? P->tidx : P->colidx,
                d ? P->tmap : nullptr, P->vals32, parts ? L.qord : L.jlev,
                parts ? L.qipos : L.ipos, parts ? L.qptr : L.pptr, nullptr, v, P->num_sms * 16, s,
                copy_diag(P, d), d ? !P->upper : P->upper);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Largest part whose unknowns fit a block's shared memory (the blocked
// kernel keeps a tile's unknowns there).
int max_part_rows(sptrsv_plan_t P) {
    const int esize = P->f64 ? 8 : 4;
    const int room = P->smem_optin - 128;
    return room > esize * 32 ? (room / esize) & ~31 : 32;
}

// The part size of the next partitioned solve: the plan's setting or the
// rows divided evenly over the SMs, at most max_part_rows.
int resolve_part_rows(sptrsv_plan_t P) {
    long long S = P->part_rows > 0 ? P->part_rows
                                   : ((long long)P->n + P->num_sms - 1) / P->num_sms;
    const int cap = max_part_rows(P);
    if (S > cap) S = cap;
    if (S < 1) S = 1;
    return (int)S;
}

// Part-ordered copy of one direction's pattern and values for the
// partitioned solve (layout in solve_parts.cu): the independent blocks of the
// substitution order and their depths, the parts (balanced pieces of long
// blocks, short blocks packed together) and their hand-out order (deepest
// block first), the level order jlev stably re-sorted by part, its inverse,
// the copy with columns renumbered to positions, its self-check (every entry
// names its own or an earlier position) and the publication buffer.
// Allocates and synchronises s.
sptrsv_status_t build_parts(sptrsv_plan_t P, bool trans, cudaStream_t s) {
    Levels& L = trans ? P->trn : P->fwd;
    const int S = resolve_part_rows(P);
    if (L.qord && L.qS == S) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    CK(cudaStreamSynchronize(s));
    free_parts(L);
    const int n = P->n, nnz = P->nnz;
    const bool upper = trans ? !P->upper : P->upper;
    const size_t esize = P->f64 ? sizeof(double) : sizeof(float);
    const int* ptr = trans ? P->tptr : P->rowptr;
    const int* idx = trans ? P->tidx : P->colidx;
    const int* vmap = trans ? P->tmap : nullptr;
    const size_t nz = nnz > 0 ? (size_t)nnz : 1;
    const size_t N = (size_t)n;
    const int hist_n = radix_hist_entries(n);
    int *qord = nullptr, *qipos = nullptr, *qptr = nullptr, *qidx = nullptr, *scratch = nullptr;
    int* qpart = nullptr;
    void *qvals = nullptr, *xq = nullptr;
    cudaError_t e = cudaMalloc(&qord, sizeof(int) * N);
    if (e == cudaSuccess) e = cudaMalloc(&qipos, sizeof(int) * N);
    if (e == cudaSuccess) e = cudaMalloc(&qptr, sizeof(int) * (N + 1));
    if (e == cudaSuccess) e = cudaMalloc(&qidx, sizeof(int) * nz);
    if (e == cudaSuccess) e = cudaMalloc(&qvals, esize * nz);
    if (e == cudaSuccess) e = cudaMalloc(&xq, esize * N);
    // scratch (ints): diff n+1, cover n+2, bflag n, bscan n+1, bstart n+1,
    // depth n, pflag n, pscan n+1, pstart n+1, pkey n, horder n, prank n,
    // psize n, rowkey n, lens n, 2 counters | radix sort: 4 n + 2 hist
    const size_t scratch_ints = 22 * N + 16 + 2 * (size_t)hist_n;
    if (e == cudaSuccess) e = cudaMalloc(&scratch, sizeof(int) * scratch_ints);
    int* diff = scratch;
    int* cover = diff + (N + 1);
    int* bflag = cover + (N + 2);
    int* bscan = bflag + N;
    int* bstart = bscan + (N + 1);
    int* depth = bstart + (N + 1);
    int* pflag = depth + N;
    int* pscan = pflag + N;
    int* pstart = pscan + (N + 1);
    int* pkey = pstart + (N + 1);
    int* horder = pkey + N;
    int* prank = horder + N;
    int* psize = prank + N;
    int* rowkey = psize + N;
    int* lens = rowkey + N;
    int* counters = lens + N;  // [0] longest part
    int* k_a = counters + 8;
    int* v_a = k_a + N;
    int* k_b = v_a + N;
    int* v_b = k_b + N;
    int* hist = v_b + N;
    int* hist_scan = hist + hist_n;
    int* piece = hist_scan + hist_n;
    int* pkey2 = piece + N;
    int* horder1 = pkey2 + N;
    int nb = 0, np = 0, maxpart = 0;
    // independent blocks: no dependency span covers their first position
    if (e == cudaSuccess) e = cudaMemsetAsync(diff, 0, sizeof(int) * (N + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(depth, 0, sizeof(int) * N, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters, 0, sizeof(int) * 8, s);
    if (e == cudaSuccess) e = launch_part_spans(n, ptr, idx, upper, diff, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(diff, cover, n + 1, s);
    if (e == cudaSuccess) e = launch_block_flags(n, cover, bflag, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(bflag, bscan, n, s);
    if (e == cudaSuccess) e = launch_flag_scatter(n, bflag, bscan, bstart, s);
    if (e == cudaSuccess) e = launch_block_depth(n, upper, L.lev, bscan, depth, s);
    // parts, numbered in order of substitution
    if (e == cudaSuccess) e = launch_part_flags(n, S, bscan, bstart, pflag, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(pflag, pscan, n, s);
    if (e == cudaSuccess) e = launch_flag_scatter(n, pflag, pscan, pstart, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nb, bscan + n, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&np, pscan + n, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && (np < 1 || np > n || nb < 1 || nb > n)) e = cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaMalloc(&qpart, sizeof(int) * ((size_t)np + 1));
    // hand-out order: latest start first -- by the block's slack (deepest
    // level minus its depth) plus the piece's share of the block's levels,
    // then order of substitution.  SPTRSV_PART_ORDER=2: by piece index (every
    // first piece, then every second piece, ...), deepest block first among
    // equal pieces; =1: deepest block first, its pieces together.
    const int maxdepth = L.nlev > 0 ? L.nlev - 1 : 0;
    const long long order = env_ll("SPTRSV_PART_ORDER", 3);
    const bool by_piece = order == 2;
    if (order == 3) {
        // latest start first: slack of the block plus the piece's share of its levels
        if (e == cudaSuccess) e = launch_part_piece(np, pstart, bscan, bstart, pscan, piece, s);
        if (e == cudaSuccess)
            e = launch_part_alap_keys(np, maxdepth, pstart, bscan, bstart, pscan, depth, piece,
                                      pkey, s);
        if (e == cudaSuccess)
            e = radix_sort_values(pkey, nullptr, np, bits_for(2 * maxdepth + 1), horder, k_a, v_a,
                                  k_b, v_b, hist, hist_scan, P->status, s);
    } else if (e == cudaSuccess) {
        e = launch_part_depth_keys(np, maxdepth, pstart, bscan, depth, pkey, s);
    }
    if (e == cudaSuccess && order != 3)
        e = radix_sort_values(pkey, nullptr, np, bits_for(maxdepth),
                              by_piece ? horder1 : horder, k_a, v_a, k_b, v_b, hist, hist_scan,
                              P->status, s);
    if (by_piece) {
        if (e == cudaSuccess) e = launch_part_piece(np, pstart, bscan, bstart, pscan, piece, s);
        if (e == cudaSuccess) e = launch_gather(piece, np, horder1, np, pkey2, P->status, s);
        if (e == cudaSuccess)
            e = radix_sort_values(pkey2, horder1, np, bits_for(np - 1), horder, k_a, v_a, k_b,
                                  v_b, hist, hist_scan, P->status, s);
    }
    if (e == cudaSuccess) e = launch_inverse_perm(horder, np, prank, s);
    if (e == cudaSuccess) e = launch_part_sizes(np, horder, pstart, psize, counters, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(psize, qpart, np, s);
    if (e == cudaSuccess) e = launch_row_part_keys(n, L.jlev, upper, pscan, prank, rowkey, s);
    // the copy: rows by part (hand-out order), by level inside a part
    if (e == cudaSuccess)
        e = radix_sort_values(rowkey, L.jlev, n, bits_for(np - 1), qord, k_a, v_a, k_b, v_b,
                              hist, hist_scan, P->status, s);
    if (e == cudaSuccess) e = launch_inverse_perm(qord, n, qipos, s);
    if (e == cudaSuccess) e = launch_ordered_lengths(n, ptr, qord, lens, s);
    if (e == cudaSuccess) e = launch_exclusive_scan(lens, qptr, n, s);
    if (e == cudaSuccess)
        e = launch_permute_rows(P->f64, n, ptr, idx, vmap, P->vals, qord, qipos, qptr, qidx,
                                qvals, P->num_sms * 16, s, copy_diag(P, trans), upper);
    if (e == cudaSuccess) e = launch_verify_permuted(n, qptr, qidx, P->status, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&maxpart, counters, sizeof(int),
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    sptrsv_status_t rc = e == cudaSuccess ? SPTRSV_OK
                         : e == cudaErrorUnknown ? SPTRSV_ERR_INTERNAL : cuda_fail(e);
    int row = -1;
    if (rc == SPTRSV_OK && take_status(P, s, &row) != SPTRSV_OK) rc = SPTRSV_ERR_INTERNAL;
    if (rc == SPTRSV_OK && (maxpart < 1 || maxpart > S)) rc = SPTRSV_ERR_INTERNAL;
    cudaFree(scratch);
    if (rc != SPTRSV_OK) {
        cudaFree(qord);
        cudaFree(qipos);
        cudaFree(qptr);
        cudaFree(qidx);
        cudaFree(qvals);
        cudaFree(xq);
        cudaFree(qpart);
        return rc;
    }
    L.qS = S;
    L.qord = qord;
    L.qipos = qipos;
    L.qptr = qptr;
    L.qidx = qidx;
    L.qvals = qvals;
    L.xq = xq;
    L.qpart = qpart;
    L.qnparts = np;
    L.qmaxpart = maxpart;
    L.qnblocks = nb;
    return SPTRSV_OK;
}

// FP32 values (gathered from the plan's FP32 copy vals32) and an FP32
// publication buffer for the level-ordered (parts = false) or part-ordered
// (parts = true) copy of an F64 plan, whose pattern must exist.  Allocates.
sptrsv_status_t build_copy_f32(sptrsv_plan_t P, bool trans, bool parts, cudaStream_t s) {
    Levels& L = trans ? P->trn : P->fwd;
    void*& vals = parts ? L.qvals32 : L.pvals32;
    void*& xpub = parts ? L.xq32 : L.xp32;
    if (vals) return SPTRSV_OK;
    if (!P->vals32 && P->nnz > 0) return SPTRSV_ERR_NOT_SUPPORTED;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    const size_t nz = P->nnz > 0 ? (size_t)P->nnz : 1;
    void *v = nullptr, *xq = nullptr;
    cudaError_t e = cudaMalloc(&v, sizeof(float) * nz);
    if (e == cudaSuccess) e = cudaMalloc(&xq, sizeof(float) * (size_t)P->n);
    if (e == cudaSuccess)
        e = launch_permute_rows(false, P->n, trans ? P->tptr : P->rowptr,
                                trans ? P->tidx : P->colidx, trans ? P->tmap : nullptr, P->vals32,
                                parts ? L.qord : L.jlev, parts ? L.qipos : L.ipos,
                                parts ? L.qptr : L.pptr, nullptr, v, P->num_sms * 16, s,
                                copy_diag(P, trans), trans ? !P->upper : P->upper);
    if (e != cudaSuccess) {
        cudaFree(v);
        cudaFree(xq);
        return cuda_fail(e);
    }
    vals = v;
    xpub = xq;
    return SPTRSV_OK;
}

sptrsv_status_t ensure_bytes(void** buf, size_t* have, size_t want, cudaStream_t s) {
    if (*have >= want) return SPTRSV_OK;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    CK(cudaStreamSynchronize(s));
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
    CK(cudaMalloc(buf, want));
    *have = want;
    return SPTRSV_OK;
}

sptrsv_status_t prof_begin(sptrsv_plan_t P, cudaStream_t s) {
    if (!P->prof) return SPTRSV_OK;
    if (P->ev.size() < 2 * (P->ev_used + 1)) {
        cudaEvent_t a, b;
        CK(cudaEventCreate(&a));
        CK(cudaEventCreate(&b));
        P->ev.push_back(a);
        P->ev.push_back(b);
    }
    CK(cudaEventRecord(P->ev[2 * P->ev_used], s));
    return SPTRSV_OK;
}

sptrsv_status_t prof_end(sptrsv_plan_t P, cudaStream_t s) {
    if (!P->prof) return SPTRSV_OK;
    CK(cudaEventRecord(P->ev[2 * P->ev_used + 1], s));
    P->ev_used++;
    return SPTRSV_OK;
}

// One triangular solve (forward pattern or transpose) of any element type:
// `f64` selects the kernels, `vals` the values they read.
// Whether a solve of this form can accumulate its published values into an
// FP64 array (SolveParams::xacc).
bool accumulates(sptrsv_algo_t algo, int nrhs) {
    if (algo == SPTRSV_ALGO_LEVEL) return false;
    return nrhs > 1 || algo == SPTRSV_ALGO_SELF || algo == SPTRSV_ALGO_SELF_PERMUTED ||
           algo == SPTRSV_ALGO_SELF_BLOCKED || algo == SPTRSV_ALGO_SELF_PARTITIONED;
}

sptrsv_status_t run_solve(sptrsv_plan_t P, bool trans, bool f64, const void* vals, const void* b,
                          long long ldb, void* x, long long ldx, int nrhs, sptrsv_algo_t algo,
                          cudaStream_t s, double* xacc = nullptr, long long ldacc = 0,
                          bool acc_first = false) {
    const bool mrhs = nrhs > 1;
    // multi-RHS solves have a launch shape of their own (sptrsv_set_mrhs_tuning);
    // a single-RHS solve takes its algorithm's shape if one was set
    const int a = (int)algo;
    const bool own = !mrhs && a >= 0 && a < 8 && P->alg_lanes[a] > 0;
    const int lanes = mrhs ? (P->mrhs_lanes ? P->mrhs_lanes : mrhs_lanes(nrhs))
                           : (own ? P->alg_lanes[a] : P->lanes);
    const int block = mrhs ? (P->mrhs_block ? P->mrhs_block : P->block)
                           : (own ? P->alg_block[a] : P->block);
    const int max_blocks = mrhs ? (P->mrhs_max_blocks >= 0 ? P->mrhs_max_blocks : P->max_blocks)
                                : (own ? P->alg_max_blocks[a] : P->max_blocks);
    if (algo == SPTRSV_ALGO_SELF_CHAINS && !mrhs) ST(build_chain(P, trans, lanes, s));
    // The copies hold the plan's element type, and FP32 values beside them
    // for the FP32 solves of a refined F64 plan (f64 != P->f64).
    const bool f32_of_f64 = !f64 && P->f64;
    if (f64 != P->f64 && !f32_of_f64) return SPTRSV_ERR_INVALID_ARG;
    const bool blocked = algo == SPTRSV_ALGO_SELF_BLOCKED && !mrhs;
    const bool permuted = (algo == SPTRSV_ALGO_SELF_PERMUTED || blocked) && !mrhs;
    if (permuted) ST(build_permuted(P, trans, s));
    if (permuted && f32_of_f64) ST(build_copy_f32(P, trans, false, s));
    const bool column = algo == SPTRSV_ALGO_SELF_COLUMN && !mrhs;
    if (column) ST(build_column(P, trans, s));
    const bool parts = algo == SPTRSV_ALGO_SELF_PARTITIONED && !mrhs;
    if (parts) ST(build_parts(P, trans, s));
    if (parts && f32_of_f64) ST(build_copy_f32(P, trans, true, s));
    // multi-RHS solves of the copying forms run on the level-ordered copy
    // (the shared-memory tiles of the blocked and partitioned forms hold one
    // column): the multi-RHS kernel with a position-ordered publication buffer
    const bool mrhs_copy = mrhs && (algo == SPTRSV_ALGO_SELF_PERMUTED ||
                                    algo == SPTRSV_ALGO_SELF_BLOCKED ||
                                    algo == SPTRSV_ALGO_SELF_PARTITIONED);
    if (mrhs_copy) {
        Levels& Lw = trans ? P->trn : P->fwd;
        ST(build_permuted(P, trans, s));
        if (f32_of_f64) ST(build_copy_f32(P, trans, false, s));
        ST(ensure_bytes(&Lw.xpm, &Lw.xpm_bytes,
                        (f64 ? sizeof(double) : sizeof(float)) * (size_t)P->n * nrhs, s));
    }
    const Levels& L = trans ? P->trn : P->fwd;
    SolveParams p;
    memset(&p, 0, sizeof(p));
    p.n = P->n;
    p.ptr = trans ? P->tptr : P->rowptr;
    p.idx = trans ? P->tidx : P->colidx;
    p.vmap = trans ? P->tmap : nullptr;
    p.vals = vals;
    p.diag_first = trans ? !P->upper : P->upper;
    p.unit = P->unit;
    p.jlev = L.jlev;
    p.b = b;
    p.ldb = ldb;
    p.x = x;
    p.ldx = ldx;
    p.nrhs = nrhs;
    p.ticket = P->counters;
    p.status = P->status;
    p.spin = P->spin;
    p.withhold = P->withhold;
    p.ipos = (algo == SPTRSV_ALGO_SELF_TILED && P->tile_level_order) ? L.ipos : nullptr;
    if (xacc && !accumulates(algo, nrhs)) return SPTRSV_ERR_INVALID_ARG;
    p.xacc = xacc;
    p.ldacc = ldacc;
    p.acc_first = acc_first ? 1 : 0;
    int launches = 0;
    if (algo == SPTRSV_ALGO_LEVEL) {
        ST(prof_begin(P, s));
        for (int m = 0; m < L.nlev; ++m) {
            p.kbeg = L.h_ilev[m];
            p.cnt = L.h_ilev[m + 1] - L.h_ilev[m];
            CK(mrhs ? launch_mrhs(f64, lanes, false, p, 0, block, s)
                    : launch_level_k1(f64, lanes, p, block, s));
        }
        ST(prof_end(P, s));
        launches = L.nlev;
    } else if (column) {
        // Alg. 4: the column structure of the system is the CSR of its
        // transpose: the plan's transposed pattern for a forward solve, the
        // caller's CSR for a transposed one.
        ColumnParams c;
        c.ptr = trans ? P->rowptr : P->tptr;
        c.idx = trans ? P->colidx : P->tidx;
        c.vmap = trans ? nullptr : P->tmap;
        c.diag_first = trans ? P->upper : !P->upper;  // a lower system
        c.count = L.count;
        c.count0 = L.count0;
        CK(launch_prep_column(f64, p, c, P->num_sms * 8, s));
        const int R = 32 / lanes;
        const long long tickets = ((long long)P->n + R - 1) / R;
        const long long want_blocks = (tickets + block / 32 - 1) / (block / 32);
        long long grid =
            (long long)column_blocks_per_sm(f64, lanes, c.vmap != nullptr, block) * P->num_sms;
        if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
        if (grid > want_blocks) grid = want_blocks;
        if (grid < 1) grid = 1;
        ST(prof_begin(P, s));
        CK(launch_column_k1(f64, lanes, p, c, (int)grid, block, s));
        ST(prof_end(P, s));
        launches = 2;
    } else if (parts) {
        // The blocked kernel on the part-ordered copy, one part per tile.
        // Rows publish to L.xq and store x(i) for the caller; b(i) is read
        // once, by row i, before x(i) is written, so in place needs no copy.
        p.ptr = L.qptr;
        p.idx = L.qidx;
        p.vmap = nullptr;
        p.vals = f32_of_f64 ? L.qvals32 : L.qvals;
        p.xp = f32_of_f64 ? L.xq32 : L.xq;
        p.prescaled = P->unit ? 0 : 1;
        p.jlev = L.qord;
        p.diag_first = 0;  // the copy stores an upper row's entries in descending order
        p.part_ptr = L.qpart;
        p.nparts = L.qnparts;
        CK(launch_prep_self(f64, P->n, 1, p.xp, 1, nullptr, 0, nullptr, P->counters,
                            P->num_sms * 8, s));
        const int cl = P->part_cluster;
        const long long groups = ((long long)L.qnparts + cl - 1) / cl;
        long long grid = blocked_resident_blocks(f64, lanes, cl, block, L.qmaxpart, P->num_sms);
        if (grid < cl) return SPTRSV_ERR_INVALID_ARG;  // this shape cannot run
        if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
        if (grid > groups * cl) grid = groups * cl;
        grid = grid / cl * cl;
        if (grid < cl) grid = cl;
        ST(prof_begin(P, s));
        CK(launch_blocked_k1(f64, lanes, p, L.qmaxpart, (int)grid, block, s, cl));
        ST(prof_end(P, s));
        launches = 2;
    } else if (mrhs_copy) {
        // Columns publish to the position-ordered buffer L.xpm ([n][nrhs]) and
        // store x(i) for the caller; every b(i, c) is read by row i before
        // x(i, c) is written, so an in-place solve needs no copy of b.
        p.ptr = L.pptr;
        p.idx = L.pidx;
        p.vmap = nullptr;
        p.diag_first = 0;  // the copy stores an upper row's entries in descending order
        p.vals = f32_of_f64 ? L.pvals32 : L.pvals;
        p.xp = L.xpm;
        p.prescaled = P->unit ? 0 : 1;
        CK(launch_prep_self(f64, P->n, nrhs, L.xpm, nrhs, nullptr, 0, nullptr, P->counters,
                            P->num_sms * 8, s));
        const int R = 32 / lanes;
        const long long tickets = ((long long)P->n + R - 1) / R;
        const long long want_blocks = (tickets + block / 32 - 1) / (block / 32);
        long long grid = (long long)self_blocks_per_sm(f64, lanes, true, false, block) * P->num_sms;
        if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
        if (grid > want_blocks) grid = want_blocks;
        if (grid < 1) grid = 1;
        ST(prof_begin(P, s));
        CK(launch_mrhs(f64, lanes, true, p, (int)grid, block, s));
        ST(prof_end(P, s));
        launches = 2;
    } else if (permuted) {
        // Rows publish to the position-ordered buffer L.xp and store x(i) for
        // the caller; b(i) is read once, by row i, before x(i) is written, so
        // an in-place solve needs no copy of b.
        p.ptr = L.pptr;
        p.idx = L.pidx;
        p.vmap = nullptr;
        p.diag_first = 0;  // the copy stores an upper row's entries in descending order
        p.vals = f32_of_f64 ? L.pvals32 : L.pvals;
        p.xp = f32_of_f64 ? L.xp32 : L.xp;
        p.prescaled = P->unit ? 0 : 1;
        CK(launch_prep_self(f64, P->n, 1, p.xp, 1, nullptr, 0, nullptr, P->counters,
                            P->num_sms * 8, s));
        const int R = 32 / lanes;
        const long long tickets = ((long long)P->n + R - 1) / R;
        const long long want_blocks = (tickets + block / 32 - 1) / (block / 32);
        if (blocked) {
            const long long tiles = ((long long)P->n + P->tile_rows - 1) / P->tile_rows;
            long long grid = blocked_resident_blocks(f64, lanes, 1, block, P->tile_rows,
                                                     P->num_sms);
            if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
            if (grid > tiles) grid = tiles;
            if (grid < 1) grid = 1;
            ST(prof_begin(P, s));
            CK(launch_blocked_k1(f64, lanes, p, P->tile_rows, (int)grid, block, s));
            ST(prof_end(P, s));
        } else {
            long long grid =
                (long long)self_perm_blocks_per_sm(f64, lanes, block) * P->num_sms;
            if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
            if (grid > want_blocks) grid = want_blocks;
            if (grid < 1) grid = 1;
            ST(prof_begin(P, s));
            CK(launch_self_k1(f64, lanes, p, (int)grid, block, s));
            ST(prof_end(P, s));
        }
        launches = 2;
    } else {
        const size_t esize = f64 ? sizeof(double) : sizeof(float);
        void* bcopy = nullptr;
        if (x == b) {  // in place: keep b aside, x becomes the publication buffer
            ST(ensure_bytes(&P->bcopy, &P->bcopy_bytes, esize * (size_t)P->n * nrhs, s));
            bcopy = P->bcopy;
            p.b = bcopy;
            p.ldb = nrhs;
        }
        CK(launch_prep_self(f64, P->n, nrhs, x, ldx, b, ldb, bcopy, P->counters,
                            P->num_sms * 8, s));
        const int R = 32 / lanes;
        const long long tickets = ((long long)P->n + R - 1) / R;
        const long long want_blocks = (tickets + block / 32 - 1) / (block / 32);
        long long grid =
            (long long)self_blocks_per_sm(f64, lanes, mrhs, trans, block) * P->num_sms;
        if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
        if (grid > want_blocks) grid = want_blocks;
        if (grid < 1) grid = 1;
        if (algo == SPTRSV_ALGO_SELF_TILED && !mrhs) {
            const long long tiles = ((long long)P->n + P->tile_rows - 1) / P->tile_rows;
            grid = (long long)tiled_blocks_per_sm(f64, lanes, trans, block, P->tile_rows) *
                   P->num_sms;
            if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
            if (grid > tiles) grid = tiles;
            if (grid < 1) grid = 1;
            ST(prof_begin(P, s));
            CK(launch_tiled_k1(f64, lanes, p, P->tile_rows, (int)grid, block, s));
            ST(prof_end(P, s));
        } else if (algo == SPTRSV_ALGO_SELF_CHAINS && !mrhs) {
            grid = (long long)chain_blocks_per_sm(f64, lanes, trans, block) * P->num_sms;
            if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
            if (grid > want_blocks) grid = want_blocks;
            if (grid < 1) grid = 1;
            ST(prof_begin(P, s));
            CK(launch_chain_k1(f64, lanes, p, L.torder[log2_lanes(lanes)], (int)grid, block,
                               s));
            ST(prof_end(P, s));
        } else {
            ST(prof_begin(P, s));
            CK(mrhs ? launch_mrhs(f64, lanes, true, p, (int)grid, block, s)
                    : launch_self_k1(f64, lanes, p, (int)grid, block, s));
            ST(prof_end(P, s));
        }
        launches = 2;
    }
    P->last_launches = launches;
    return SPTRSV_OK;
}

sptrsv_status_t solve_common(sptrsv_plan_t P, bool trans, const void* b, void* x, int nrhs,
                             int ld, sptrsv_algo_t algo, void* stream) {
    if (!P || nrhs < 1 || ld < nrhs ||
        (algo != SPTRSV_ALGO_LEVEL && algo != SPTRSV_ALGO_SELF && algo != SPTRSV_ALGO_SELF_TILED &&
         algo != SPTRSV_ALGO_SELF_CHAINS && algo != SPTRSV_ALGO_SELF_PERMUTED &&
         algo != SPTRSV_ALGO_SELF_COLUMN && algo != SPTRSV_ALGO_SELF_BLOCKED &&
         algo != SPTRSV_ALGO_SELF_PARTITIONED && algo != SPTRSV_ALGO_AUTO))
        return SPTRSV_ERR_INVALID_ARG;
    if (algo == SPTRSV_ALGO_AUTO) algo = P->default_algo;
    P->last_launches = 0;
    if (P->n == 0) return SPTRSV_OK;
    if (!b || !x) return SPTRSV_ERR_INVALID_ARG;
    DeviceGuard g(P->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (trans) ST(build_transpose(P, s));
    return run_solve(P, trans, P->f64, P->vals, b, ld, x, ld, nrhs, algo, s);
}

}  // namespace

extern "C" {

sptrsv_status_t sptrsv_analyze(int n, int nnz, const int* d_rowptr, const int* d_colidx,
                               const void* d_vals, sptrsv_dtype_t dtype, sptrsv_uplo_t uplo,
                               sptrsv_diag_t diag, void* stream, sptrsv_plan_t* plan) {
    g_last_error_row = -1;
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    *plan = nullptr;
    if (n < 0 || nnz < 0 || (dtype != SPTRSV_F64 && dtype != SPTRSV_F32) ||
        (uplo != SPTRSV_LOWER && uplo != SPTRSV_UPPER) ||
        (diag != SPTRSV_NON_UNIT && diag != SPTRSV_UNIT))
        return SPTRSV_ERR_INVALID_ARG;
    // a lane's cursor over a row's entries runs up to 32 x kChunk entries
    // past the row's end: below SPTRSV_MAX_SIZE it stays an int
    static_assert(32 * kChunk <= 2147483647 - SPTRSV_MAX_SIZE, "cursor headroom");
    if (n > SPTRSV_MAX_SIZE || nnz > SPTRSV_MAX_SIZE) return SPTRSV_ERR_INVALID_ARG;
    if (n > 0 && (!d_rowptr || (nnz > 0 && (!d_colidx || !d_vals)))) return SPTRSV_ERR_INVALID_ARG;
    if (n > 0 && nnz == 0 && diag == SPTRSV_NON_UNIT) {
        g_last_error_row = 0;
        return SPTRSV_ERR_ZERO_PIVOT;
    }
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    sptrsv_plan_t P = new sptrsv_plan_s();
    cudaError_t e = cudaGetDevice(&P->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, P->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&P->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                   P->device);
    if (e != cudaSuccess) {
        destroy(P);
        return cuda_fail(e);
    }
    P->n = n;
    P->nnz = nnz;
    P->f64 = dtype == SPTRSV_F64;
    P->upper = uplo == SPTRSV_UPPER;
    P->unit = diag == SPTRSV_UNIT;
    P->rowptr = d_rowptr;
    P->colidx = d_colidx;
    P->vals = d_vals;
    P->lanes = default_lanes(n, nnz);
    P->max_blocks = 2 * P->num_sms;
    P->spin.limit = env_ll("SPTRSV_SPIN_LIMIT", 1ll << 24);
    P->spin.hot = (int)env_ll("SPTRSV_SPIN_HOT", 256);
    P->spin.max_ns = (unsigned)env_ll("SPTRSV_SPIN_MAX_NS", 128);
    sptrsv_status_t rc = SPTRSV_OK;
    e = cudaMalloc(&P->counters, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&P->status, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(P->counters, 0, 4 * sizeof(int), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->status, 0xff, sizeof(unsigned long long), s);
    if (e != cudaSuccess) rc = cuda_fail(e);
    if (rc == SPTRSV_OK && n > 0) {
        e = launch_validate(n, nnz, d_rowptr, d_colidx, d_vals, P->f64, P->upper, P->unit,
                            P->status, P->num_sms * 32, s);
        if (e != cudaSuccess) rc = cuda_fail(e);
        int row = -1;
        if (rc == SPTRSV_OK) rc = take_status(P, s, &row);
        if (rc == SPTRSV_ERR_STRUCTURE || rc == SPTRSV_ERR_ZERO_PIVOT) g_last_error_row = row;
        // Setup (Table 1): the transposed pattern (TRANS_GPU; also the column
        // structure of the transposed and column-wise solves), then the
        // levels by the automatic method: Kahn's algorithm in one launch,
        // falling back to the sweep on deep, narrow graphs.
        if (rc == SPTRSV_OK) rc = build_transpose_pattern(P, s);
        if (rc == SPTRSV_OK)
            rc = build_levels(P, d_rowptr, d_colidx, P->upper, P->fwd, s, SPTRSV_ANALYSIS_AUTO,
                              P->tptr, P->tidx);
    }
    if (rc != SPTRSV_OK) {
        destroy(P);
        return rc;
    }
    P->analysis_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *plan = P;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_reanalyze(sptrsv_plan_t plan, int transpose, sptrsv_analysis_t method,
                                 void* stream) {
    if (!plan || (transpose != 0 && transpose != 1) ||
        (method != SPTRSV_ANALYSIS_SWEEP && method != SPTRSV_ANALYSIS_KAHN_HOST_LOOP &&
         method != SPTRSV_ANALYSIS_KAHN_PERSISTENT && method != SPTRSV_ANALYSIS_AUTO))
        return SPTRSV_ERR_INVALID_ARG;
    sptrsv_plan_t P = plan;
    if (P->n == 0) return SPTRSV_OK;
    DeviceGuard g(P->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    if (transpose) ST(build_transpose(P, s));
    CK(cudaStreamSynchronize(s));
    const auto t0 = std::chrono::steady_clock::now();
    const bool kahn = method != SPTRSV_ANALYSIS_SWEEP;
    // Kahn's algorithm walks the outgoing edges: the transposed pattern for
    // the forward system (built here if needed, as Table 1's TRANS_GPU), the
    // caller's CSR for the transposed one.
    if (kahn && !transpose) ST(build_transpose_pattern(P, s));
    Levels& L = transpose ? P->trn : P->fwd;
    Levels fresh;
    const int* ptr = transpose ? P->tptr : P->rowptr;
    const int* idx = transpose ? P->tidx : P->colidx;
    const bool upper = transpose ? !P->upper : P->upper;
    sptrsv_status_t rc = build_levels(P, ptr, idx, upper, fresh, s, method,
                                      transpose ? P->rowptr : P->tptr,
                                      transpose ? P->colidx : P->tidx);
    if (rc != SPTRSV_OK) {
        free_levels(fresh);
        return rc;
    }
    P->analysis_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    (void)kahn;
    // Levels are unique, so data derived from them stay valid; keep the
    // segment orders and counters, rebuild the level-ordered copy lazily.
    for (int k = 0; k < 6; ++k) {
        fresh.torder[k] = L.torder[k];
        fresh.nslev[k] = L.nslev[k];
        L.torder[k] = nullptr;
    }
    fresh.count0 = L.count0;
    fresh.count = L.count;
    L.count0 = L.count = nullptr;
    free_levels(L);
    L = std::move(fresh);
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_analysis_method(sptrsv_plan_t plan, int transpose, int* method) {
    if (!plan || !method || (transpose != 0 && transpose != 1)) return SPTRSV_ERR_INVALID_ARG;
    if (transpose && !plan->has_trans && plan->n > 0) return SPTRSV_ERR_NOT_SUPPORTED;
    *method = (transpose ? plan->trn : plan->fwd).method;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_free(sptrsv_plan_t plan) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    {
        DeviceGuard g(plan->device);
        cudaDeviceSynchronize();
    }
    destroy(plan);
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_solve(sptrsv_plan_t plan, const void* d_b, void* d_x, int nrhs, int ld,
                             sptrsv_algo_t algo, void* stream) {
    return solve_common(plan, false, d_b, d_x, nrhs, ld, algo, stream);
}

sptrsv_status_t sptrsv_solve_transpose(sptrsv_plan_t plan, const void* d_b, void* d_x, int nrhs,
                                       int ld, sptrsv_algo_t algo, void* stream) {
    return solve_common(plan, true, d_b, d_x, nrhs, ld, algo, stream);
}

sptrsv_status_t sptrsv_prepare_transpose(sptrsv_plan_t plan, void* stream) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    if (plan->n == 0) return SPTRSV_OK;
    DeviceGuard g(plan->device);
    return build_transpose(plan, (cudaStream_t)stream);
}

sptrsv_status_t sptrsv_prepare(sptrsv_plan_t plan, int transpose, sptrsv_algo_t algo,
                               void* stream) {
    if (!plan || (transpose != 0 && transpose != 1) || (int)algo < SPTRSV_ALGO_LEVEL ||
        (int)algo > SPTRSV_ALGO_AUTO)
        return SPTRSV_ERR_INVALID_ARG;
    sptrsv_plan_t P = plan;
    if (P->n == 0) return SPTRSV_OK;
    DeviceGuard g(P->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    if (algo == SPTRSV_ALGO_AUTO) algo = P->default_algo;
    const bool trans = transpose != 0;
    if (trans) ST(build_transpose(P, s));
    const int a = (int)algo;
    const int lanes = P->alg_lanes[a] > 0 ? P->alg_lanes[a] : P->lanes;
    switch (algo) {
        case SPTRSV_ALGO_SELF_CHAINS: ST(build_chain(P, trans, lanes, s)); break;
        case SPTRSV_ALGO_SELF_PERMUTED:
        case SPTRSV_ALGO_SELF_BLOCKED: ST(build_permuted(P, trans, s)); break;
        case SPTRSV_ALGO_SELF_PARTITIONED: ST(build_parts(P, trans, s)); break;
        case SPTRSV_ALGO_SELF_COLUMN: ST(build_column(P, trans, s)); break;
        default: break;
    }
    CK(cudaStreamSynchronize(s));
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_grad_vals(sptrsv_plan_t plan, const void* d_y, const void* d_x, int nrhs,
                                 int ld, void* d_gvals, void* stream) {
    if (!plan || nrhs < 1 || ld < nrhs) return SPTRSV_ERR_INVALID_ARG;
    if (plan->n == 0) return SPTRSV_OK;
    if (!d_y || !d_x || (plan->nnz > 0 && !d_gvals)) return SPTRSV_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    CK(launch_grad_vals(plan->f64, plan->lanes, plan->n, plan->rowptr, plan->colidx, plan->unit,
                        d_y, ld, d_x, ld, nrhs, d_gvals, (cudaStream_t)stream,
                        plan->num_sms * 16));
    plan->last_launches = 1;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_residual(sptrsv_plan_t plan, const double* d_b, const double* d_x,
                                double* d_r, int nrhs, int ld, void* stream) {
    if (!plan || nrhs < 1 || ld < nrhs) return SPTRSV_ERR_INVALID_ARG;
    if (!plan->f64) return SPTRSV_ERR_NOT_SUPPORTED;
    if (plan->n == 0) return SPTRSV_OK;
    if (!d_b || !d_x || !d_r) return SPTRSV_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    CK(launch_residual(plan->n, plan->nnz, plan->rowptr, plan->colidx,
                       (const double*)plan->vals, plan->unit, nrhs, d_b, ld, d_x, ld, d_r, ld,
                       nullptr, nullptr, false, plan->num_sms * 16, (cudaStream_t)stream));
    plan->last_launches = 1;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_refresh_values(sptrsv_plan_t plan, void* stream) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    if (plan->nnz == 0) return SPTRSV_OK;
    DeviceGuard g(plan->device);
    if (plan->vals32)
        CK(launch_to_f32(plan->nnz, 1, (const double*)plan->vals, 1, plan->vals32, nullptr,
                         plan->num_sms * 16, (cudaStream_t)stream));
    CK(refresh_permuted(plan, (cudaStream_t)stream));
    plan->anorm = -1.0;  // the refined solve measures ||A||_inf again
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_values(sptrsv_plan_t plan, const void* d_vals, void* stream) {
    if (!plan || (plan->nnz > 0 && !d_vals)) return SPTRSV_ERR_INVALID_ARG;
    plan->vals = d_vals;
    return sptrsv_refresh_values(plan, stream);
}

// Refinement of one right-hand side in passes of the one-pass kernel
// (refine.cu): the first pass solves from x = 0 and applies K corrections in
// the same sweep; the host then reads the residual norm of every step and,
// if none met `tol` and corrections remain, runs another pass from the
// current x.  Needs the level-ordered copy and its FP32 values.
sptrsv_status_t refine_in_passes(sptrsv_plan_t P, const double* d_b, double* d_x, long long ld,
                                 int max_iter, double tol, int* iters, double* rel_resid,
                                 cudaStream_t s) {
    const int n = P->n;
    const int grid16 = P->num_sms * 16;
    ST(build_permuted(P, false, s));
    ST(build_copy_f32(P, false, false, s));
    const Levels& L = P->fwd;
    const int S = kRefineMaxSteps + 1;
    const size_t want = (size_t)S * n;
    if (!P->rf_dpub || P->rf_bytes < want) {
        CK(cudaStreamSynchronize(s));
        cudaFree(P->rf_dpub);
        cudaFree(P->rf_xpub);
        P->rf_dpub = P->rf_xpub = nullptr;
        P->rf_bytes = 0;
        CK(cudaMalloc(&P->rf_dpub, sizeof(float) * want));
        CK(cudaMalloc(&P->rf_xpub, sizeof(double) * want));
        P->rf_bytes = want;
    }
    if (!P->rf_norms) CK(cudaMalloc(&P->rf_norms, 2 * S * sizeof(unsigned long long)));
    if (!P->stats) CK(cudaMalloc(&P->stats, 4 * sizeof(unsigned long long)));
    int launches = 0;
    if (P->anorm < 0.0) {  // ||A||_inf of the current values, once
        CK(cudaMemsetAsync(P->stats, 0, 4 * sizeof(unsigned long long), s));
        CK(launch_residual(n, P->nnz, P->rowptr, P->colidx, (const double*)P->vals, P->unit, 1,
                           d_b, ld, d_b, ld, nullptr, 0, nullptr, P->stats, true, grid16, s));
        launches += 1;
        unsigned long long h = 0;
        CK(cudaMemcpyAsync(&h, P->stats + 1, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        memcpy(&P->anorm, &h, sizeof(double));
    }
    // launch shape: the level-ordered form's (its tuned width), blocks of at most 512
    const int a = (int)SPTRSV_ALGO_SELF_PERMUTED;
    const int lanes = P->alg_lanes[a] > 0 ? P->alg_lanes[a] : P->lanes;
    int block = P->alg_lanes[a] > 0 ? P->alg_block[a] : P->block;
    if (block > 512) block = 512;
    const int max_blocks = P->alg_lanes[a] > 0 ? P->alg_max_blocks[a] : P->max_blocks;
    const int R = 32 / lanes;
    const long long want_blocks = (((long long)n + R - 1) / R + block / 32 - 1) / (block / 32);
    long long grid = (long long)refine_blocks_per_sm(lanes, block) * P->num_sms;
    if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
    if (grid > want_blocks) grid = want_blocks;
    if (grid < 1) grid = 1;
    RefineParams r;
    memset(&r, 0, sizeof(r));
    r.n = n;
    r.ptr = L.pptr;
    r.idx = L.pidx;
    r.v64 = (const double*)L.pvals;
    r.v32 = (const float*)L.pvals32;
    r.jlev = L.jlev;
    r.unit = P->unit;
    r.diag_first = 0;  // the copy stores an upper row's entries in descending order
    r.b = d_b;
    r.ldb = ld;
    r.x = d_x;
    r.ldx = ld;
    r.dpub = (float*)P->rf_dpub;
    r.xpub = (double*)P->rf_xpub;
    r.ticket = P->counters;
    r.status = P->status;
    r.rmax = P->rf_norms;
    r.xmax = P->rf_norms + S;
    r.spin = P->spin;
    int applied = 0;
    double rel = 0.0, bmax = 0.0;
    for (bool first = true;; first = false) {
        // a first pass takes three corrections: FP32 solves of a well-
        // conditioned system reach FP64 accuracy after two, and the residual
        // a pass measures last is that of its next-to-last iterate; later
        // passes take the rest, at most kRefineMaxSteps steps each
        const int left = max_iter - applied;
        r.has_init = first ? 0 : 1;
        r.K = first ? (left < 3 ? left : 3)
                    : (left - 1 < kRefineMaxSteps ? left - 1 : kRefineMaxSteps);
        CK(cudaMemsetAsync(P->rf_norms, 0, 2 * S * sizeof(unsigned long long), s));
        CK(launch_refine_pass(lanes, r, (int)grid, block, s));
        launches += 2;
        unsigned long long h[2 * (kRefineMaxSteps + 1)];
        CK(cudaMemcpyAsync(h, P->rf_norms, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double nr[2 * (kRefineMaxSteps + 1)];
        memcpy(nr, h, sizeof(nr));
        if (first) bmax = nr[0];  // step 0 of the first pass: r^0 = b
        applied += first ? r.K : r.K + 1;
        bool met = false;
        for (int m = first ? 1 : 0; m <= r.K; ++m) {
            const double denom = bmax + P->anorm * nr[S + m];
            rel = denom > 0.0 ? nr[m] / denom : (nr[m] > 0.0 ? INFINITY : 0.0);
            met = met || rel <= tol;
        }
        if (met || applied >= max_iter) break;
    }
    if (iters) *iters = applied;
    if (rel_resid) *rel_resid = rel;
    P->last_launches = launches;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_solve_refined(sptrsv_plan_t plan, const double* d_b, double* d_x,
                                     int nrhs, int ld, int max_iter, double tol, int* iters,
                                     double* rel_resid, void* stream) {
    if (!plan || nrhs < 1 || ld < nrhs || max_iter < 0 || !(tol >= 0.0))
        return SPTRSV_ERR_INVALID_ARG;
    if (!plan->f64) return SPTRSV_ERR_NOT_SUPPORTED;
    if (iters) *iters = 0;
    if (rel_resid) *rel_resid = 0.0;
    if (plan->n == 0) return SPTRSV_OK;
    if (!d_b || !d_x || d_b == d_x) return SPTRSV_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return SPTRSV_ERR_NOT_SUPPORTED;
    sptrsv_plan_t P = plan;
    const int n = P->n;
    const int grid = P->num_sms * 16;
    if (!P->vals32 && P->nnz > 0) {
        CK(cudaMalloc(&P->vals32, sizeof(float) * (size_t)P->nnz));
        CK(launch_to_f32(P->nnz, 1, (const double*)P->vals, 1, P->vals32, nullptr, grid, s));
    }
    const size_t need = (size_t)n * nrhs;
    if (P->rd_elems < need) {
        CK(cudaStreamSynchronize(s));
        cudaFree(P->r32);
        cudaFree(P->d32);
        P->r32 = P->d32 = nullptr;
        P->rd_elems = 0;
        CK(cudaMalloc(&P->r32, sizeof(float) * need));
        CK(cudaMalloc(&P->d32, sizeof(float) * need));
        P->rd_elems = need;
    }
    if (!P->stats) CK(cudaMalloc(&P->stats, 4 * sizeof(unsigned long long)));
    CK(cudaMemsetAsync(P->stats, 0, 4 * sizeof(unsigned long long), s));
    // One right-hand side in the one-pass form: every step in one sweep.
    if (nrhs == 1 && max_iter >= 1 && P->refine_mode == SPTRSV_REFINE_ONE_PASS)
        return refine_in_passes(P, d_b, d_x, ld, max_iter, tol, iters, rel_resid, s);
    // The FP32 solves run the plan's default form (sptrsv_set_default_algo,
    // e.g. the autotuner's choice) with that form's launch shape.  The forms
    // that can accumulate add each published correction straight into the
    // FP64 solution x (no separate update pass); the others store it in an
    // FP32 vector that an update pass adds.
    const sptrsv_algo_t algo = P->default_algo;
    const bool fused = accumulates(algo, nrhs);
    int launches = 0;
    auto correction = [&](bool first) -> sptrsv_status_t {
        if (fused) {
            ST(run_solve(P, false, false, P->vals32, P->r32, nrhs, P->d32, nrhs, nrhs, algo, s,
                         d_x, ld, first));
            launches += P->last_launches;
        } else {
            ST(run_solve(P, false, false, P->vals32, P->r32, nrhs, P->d32, nrhs, nrhs, algo, s));
            launches += P->last_launches;
            CK(launch_update(n, nrhs, d_x, ld, P->d32, first, nullptr, grid, s));
            launches += 1;
        }
        return SPTRSV_OK;
    };
    // x0 = 0, so r0 = b: the first FP32 solve is of b itself.
    CK(launch_to_f32(n, nrhs, d_b, ld, P->r32, P->stats + 3, grid, s));
    launches += 1;
    ST(correction(true));
    int it = 0;
    double rel = 0.0;
    if (max_iter >= 1) {
        // An FP32 solve alone does not reach the FP64 stop rule: the first
        // correction follows without reading the residual norm (one host
        // round trip fewer; with b = 0 it adds a zero correction).
        CK(launch_residual(n, P->nnz, P->rowptr, P->colidx, (const double*)P->vals, P->unit,
                           nrhs, d_b, ld, d_x, ld, nullptr, 0, P->r32, nullptr, false, grid, s));
        launches += 1;
        ST(correction(false));
        it = 1;
    }
    for (;;) {
        // r = b - A x in FP64, its FP32 copy (the next right-hand side),
        // max|r|, max|x| and, once per set of values, ||A||_inf, in one pass
        const bool want_norm = P->anorm < 0.0;
        CK(cudaMemsetAsync(P->stats, 0, 3 * sizeof(unsigned long long), s));
        CK(launch_residual(n, P->nnz, P->rowptr, P->colidx, (const double*)P->vals, P->unit,
                           nrhs, d_b, ld, d_x, ld, nullptr, 0, P->r32, P->stats, want_norm, grid,
                           s));
        launches += 1;
        unsigned long long h[4];
        CK(cudaMemcpyAsync(h, P->stats, sizeof(h), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        double st[4];
        memcpy(st, h, sizeof(st));
        if (want_norm) P->anorm = st[1];  // kept until the values change
        else st[1] = P->anorm;
        const double denom = st[3] + st[1] * st[2];
        rel = denom > 0.0 ? st[0] / denom : (st[0] > 0.0 ? INFINITY : 0.0);
        if (rel <= tol || it >= max_iter) break;
        ST(correction(false));
        ++it;
    }
    if (iters) *iters = it;
    if (rel_resid) *rel_resid = rel;
    P->last_launches = launches;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_refine_mode(sptrsv_plan_t plan, sptrsv_refine_t mode) {
    if (!plan || (mode != SPTRSV_REFINE_STAGED && mode != SPTRSV_REFINE_ONE_PASS))
        return SPTRSV_ERR_INVALID_ARG;
    plan->refine_mode = mode;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_get_refine_mode(sptrsv_plan_t plan, int* mode) {
    if (!plan || !mode) return SPTRSV_ERR_INVALID_ARG;
    *mode = (int)plan->refine_mode;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_default_algo(sptrsv_plan_t plan, sptrsv_algo_t algo) {
    const int a = (int)algo;
    if (!plan || a < SPTRSV_ALGO_LEVEL || a > SPTRSV_ALGO_SELF_PARTITIONED)
        return SPTRSV_ERR_INVALID_ARG;
    plan->default_algo = algo;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_get_default_algo(sptrsv_plan_t plan, int* algo) {
    if (!plan || !algo) return SPTRSV_ERR_INVALID_ARG;
    *algo = (int)plan->default_algo;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_tuning(sptrsv_plan_t plan, int lanes_per_row, int block_size,
                                  int max_blocks) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    const int w = lanes_per_row;
    if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32)) return SPTRSV_ERR_INVALID_ARG;
    if (block_size < 32 || block_size > 1024 || block_size % 32 != 0 || max_blocks < 0)
        return SPTRSV_ERR_INVALID_ARG;
    plan->lanes = w;
    plan->block = block_size;
    plan->max_blocks = max_blocks;
    for (int a = 0; a < 8; ++a) plan->alg_lanes[a] = 0;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_algo_tuning(sptrsv_plan_t plan, sptrsv_algo_t algo, int lanes_per_row,
                                       int block_size, int max_blocks) {
    const int a = (int)algo;
    if (!plan || a < SPTRSV_ALGO_LEVEL || a > SPTRSV_ALGO_SELF_PARTITIONED)
        return SPTRSV_ERR_INVALID_ARG;
    const int w = lanes_per_row;
    if (w == 0) {
        plan->alg_lanes[a] = 0;
        return SPTRSV_OK;
    }
    if (!(w == 1 || w == 2 || w == 4 || w == 8 || w == 16 || w == 32)) return SPTRSV_ERR_INVALID_ARG;
    if (block_size < 32 || block_size > 1024 || block_size % 32 != 0 || max_blocks < 0)
        return SPTRSV_ERR_INVALID_ARG;
    plan->alg_lanes[a] = w;
    plan->alg_block[a] = block_size;
    plan->alg_max_blocks[a] = max_blocks;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_mrhs_tuning(sptrsv_plan_t plan, int lanes_per_row, int block_size,
                                       int max_blocks) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    const int w = lanes_per_row;
    if (!(w == 0 || w == 4 || w == 8 || w == 16 || w == 32)) return SPTRSV_ERR_INVALID_ARG;
    if (block_size != 0 && (block_size < 32 || block_size > 1024 || block_size % 32 != 0))
        return SPTRSV_ERR_INVALID_ARG;
    if (max_blocks < -1) return SPTRSV_ERR_INVALID_ARG;
    plan->mrhs_lanes = w;
    plan->mrhs_block = block_size;
    plan->mrhs_max_blocks = max_blocks;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_get_tuning(sptrsv_plan_t plan, int* lanes_per_row, int* block_size,
                                  int* max_blocks) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    if (lanes_per_row) *lanes_per_row = plan->lanes;
    if (block_size) *block_size = plan->block;
    if (max_blocks) *max_blocks = plan->max_blocks;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_tiling(sptrsv_plan_t plan, int tile_rows, int level_order) {
    if (!plan || tile_rows < 32 || (level_order != 0 && level_order != 1))
        return SPTRSV_ERR_INVALID_ARG;
    const size_t esize = plan->f64 ? sizeof(double) : sizeof(float);
    if (esize * (size_t)tile_rows > 48 * 1024 - 256) return SPTRSV_ERR_INVALID_ARG;
    plan->tile_rows = tile_rows;
    plan->tile_level_order = level_order != 0;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_partition(sptrsv_plan_t plan, int part_rows, int cluster_blocks) {
    const int c = cluster_blocks;
    if (!plan || part_rows < 0 || !(c == 0 || c == 1 || c == 2 || c == 4 || c == 8))
        return SPTRSV_ERR_INVALID_ARG;
    plan->part_rows = part_rows;
    plan->part_cluster = c > 1 ? c : 1;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_get_partition(sptrsv_plan_t plan, int* part_rows, int* cluster_blocks) {
    if (!plan || !part_rows || !cluster_blocks) return SPTRSV_ERR_INVALID_ARG;
    *part_rows = resolve_part_rows(plan);
    *cluster_blocks = plan->part_cluster;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_partition_info(sptrsv_plan_t plan, int transpose, int* nparts,
                                      int* nblocks, int* max_part_rows, const int** d_part_ptr,
                                      const int** d_order) {
    if (!plan || (transpose != 0 && transpose != 1)) return SPTRSV_ERR_INVALID_ARG;
    const Levels& L = transpose ? plan->trn : plan->fwd;
    if (!L.qord && plan->n > 0) return SPTRSV_ERR_NOT_SUPPORTED;
    if (nparts) *nparts = L.qnparts;
    if (nblocks) *nblocks = L.qnblocks;
    if (max_part_rows) *max_part_rows = L.qmaxpart;
    if (d_part_ptr) *d_part_ptr = L.qpart;
    if (d_order) *d_order = L.qord;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_set_spin_limit(sptrsv_plan_t plan, long long polls) {
    if (!plan || polls < 1) return SPTRSV_ERR_INVALID_ARG;
    plan->spin.limit = polls;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_levels(sptrsv_plan_t plan, int transpose, int* nlev, const int** d_lev,
                              const int** d_ilev, const int** d_jlev) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    if (transpose && !plan->has_trans && plan->n > 0) return SPTRSV_ERR_NOT_SUPPORTED;
    const Levels& L = transpose ? plan->trn : plan->fwd;
    if (nlev) *nlev = L.nlev;
    if (d_lev) *d_lev = L.lev;
    if (d_ilev) *d_ilev = L.ilev;
    if (d_jlev) *d_jlev = L.jlev;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_transpose_pattern(sptrsv_plan_t plan, const int** d_tptr,
                                         const int** d_tidx, const int** d_tmap) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    if (!plan->has_trans && plan->n > 0) return SPTRSV_ERR_NOT_SUPPORTED;
    if (d_tptr) *d_tptr = plan->tptr;
    if (d_tidx) *d_tidx = plan->tidx;
    if (d_tmap) *d_tmap = plan->tmap;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_status(sptrsv_plan_t plan, void* stream, int* error_row) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    return take_status(plan, (cudaStream_t)stream, error_row);
}

int sptrsv_last_error_row(void) { return g_last_error_row; }

const char* sptrsv_status_string(sptrsv_status_t status) {
    switch (status) {
        case SPTRSV_OK: return "SPTRSV_OK";
        case SPTRSV_ERR_INVALID_ARG: return "SPTRSV_ERR_INVALID_ARG";
        case SPTRSV_ERR_STRUCTURE: return "SPTRSV_ERR_STRUCTURE";
        case SPTRSV_ERR_ZERO_PIVOT: return "SPTRSV_ERR_ZERO_PIVOT";
        case SPTRSV_ERR_CUDA: return "SPTRSV_ERR_CUDA";
        case SPTRSV_ERR_OOM: return "SPTRSV_ERR_OOM";
        case SPTRSV_ERR_TIMEOUT: return "SPTRSV_ERR_TIMEOUT";
        case SPTRSV_ERR_NOT_SUPPORTED: return "SPTRSV_ERR_NOT_SUPPORTED";
        case SPTRSV_ERR_INTERNAL: return "SPTRSV_ERR_INTERNAL";
    }
    return "SPTRSV_ERR_UNKNOWN";
}

const char* sptrsv_last_cuda_error(void) { return g_last_cuda; }

sptrsv_status_t sptrsv_analysis_ms(sptrsv_plan_t plan, double* ms) {
    if (!plan || !ms) return SPTRSV_ERR_INVALID_ARG;
    *ms = plan->analysis_ms;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_profile_enable(sptrsv_plan_t plan, int enable) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    plan->prof = enable != 0;
    return SPTRSV_OK;
}

sptrsv_status_t sptrsv_profile_read(sptrsv_plan_t plan, double* total_ms, int* count) {
    if (!plan) return SPTRSV_ERR_INVALID_ARG;
    DeviceGuard g(plan->device);
    double tot = 0.0;
    for (size_t k = 0; k < plan->ev_used; ++k) {
        CK(cudaEventSynchronize(plan->ev[2 * k + 1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, plan->ev[2 * k], plan->ev[2 * k + 1]));
        tot += ms;
    }
    if (total_ms) *total_ms = tot;
    if (count) *count = (int)plan->ev_used;
    plan->ev_used = 0;
    return SPTRSV_OK;
}

int sptrsv_last_launch_count(sptrsv_plan_t plan) { return plan ? plan->last_launches : 0; }

sptrsv_status_t sptrsv_debug_withhold_row(sptrsv_plan_t plan, int row) {
    if (!plan || row < -1 || row >= plan->n) return SPTRSV_ERR_INVALID_ARG;
    plan->withhold = row;
    return SPTRSV_OK;
}

}  // extern "C"
