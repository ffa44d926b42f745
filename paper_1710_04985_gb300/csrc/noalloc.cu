// Allocation-free triangular solve: sptrsv_solve_noalloc.
//
// Who needs it: callers that may not call cudaMalloc/cudaFree -- for example
// code that runs inside an embedding application which owns every byte of
// device memory through its own pool, or latency-critical loops that must
// not hit the device allocator (cudaMalloc and cudaFree can take global
// locks and synchronise the device).  They cannot build a plan (analysis
// allocates the level sets), so this entry point needs none: it validates the
// matrix and solves it in substitution order in the same stream, and keeps
// all of its working memory in one array that the library declares at file
// scope and that lives as long as the library is loaded.
//
// The working memory: a 256-byte header (ticket counter, status word) and one
// ready flag per row, for at most SPTRSV_NOALLOC_MAX_ROWS rows.  Every call
// uses the same array and leaves its contents behind; each call clears the
// header and the flags of its own rows before anything reads them.  Two calls
// whose work overlaps on the GPU (different streams, or the same array reached
// from two host threads) race on that array and give wrong results.
#include <atomic>
#include <cstdlib>
#include <mutex>

#include "internal.h"
#include "sptrsv.h"

namespace sptrsv {

namespace {

constexpr size_t kHeaderBytes = 256;

// The one scratch array: header + int flags[SPTRSV_NOALLOC_MAX_ROWS].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kHeaderBytes +
                                                                 sizeof(int) * (size_t)SPTRSV_NOALLOC_MAX_ROWS];

struct Header {
    int ticket;
    int pad;
    unsigned long long status;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void noalloc_clear_k(unsigned char* scratch, int n) {
    Header* h = (Header*)scratch;
    int* flags = (int*)(scratch + kHeaderBytes);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        flags[i] = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        h->ticket = 0;
        h->status = kStatusClear;
    }
}

// Self-scheduled solve in substitution order (no level sets).  A warp takes
// 32/W consecutive rows per ticket; a dependency on an earlier ticket waits
// for that row's ready flag (acquire) and then reads x; a dependency inside
// the ticket is forwarded by shuffle from the lane that owns the row.  x may
// alias b: a row reads its own b before it writes its own x, and nobody reads
// x(j) before flag(j) is set.  Nothing runs if validation reported an error.
template <typename T, int W>
__global__ void __launch_bounds__(1024)
    noalloc_solve_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                    const T* __restrict__ vals, int upper, int unit, const T* b, T* x,
                    unsigned char* scratch, SpinPolicy sp, int withhold) {
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    Header* h = (Header*)scratch;
    int* flags = (int*)(scratch + kHeaderBytes);
    if (ld_relaxed((const int*)&h->status) != -1 || ld_relaxed(((const int*)&h->status) + 1) != -1)
        return;  // validation failed
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    int t = 0;
    if (lane == 0) t = atomicAdd(&h->ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while ((long long)t * R < n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(&h->ticket, 1);
        const int first = (int)((long long)t * R);
        const int rows = (n - first) < R ? (n - first) : R;
        const bool has_row = grp < rows;
        const int i0 = upper ? n - 1 - first : first;
        int i = 0, beg = 0, end = 0;
        T bi = T(0), dinv = T(1);
        if (has_row) {
            i = upper ? i0 - grp : i0 + grp;
            beg = ptr[i];
            end = ptr[i + 1];
            if (sl == 0) {
                bi = b[i];
                if (!unit) dinv = T(1) / vals[upper ? beg : end - 1];
            }
        }
        int q0 = beg + sl;
        int c[E];
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
                    const int cc = idx[q];
                    if (cc != i) {
                        c[e] = cc;
                        a[e] = vals[q];
                        live |= 1u << e;
                        const int g2 = upper ? i0 - cc : cc - i0;
                        if (g2 >= 0 && g2 < grp) local |= 1u << e;
                    }
                }
            }
            pend = live;
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (((live & ~local) & (1u << e)) && ld_acquire(flags + c[e]) != 0) {
                    v[e] = ld_relaxed(x + c[e]);
                    pend &= ~(1u << e);
                }
        };
        bool lane_done = q0 >= end;
        if (!lane_done) load_chunk();
        bool published = !has_row;
        T pubv = T(0);
        T sum = T(0);
        long long waits = 0;
        unsigned ns = 32;
        while (true) {
            if (!lane_done && pend == 0) {
                const int hi = 32 - __clz(live);  // stop after the last live slot
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e >= hi) break;
                    if (live & (1u << e)) sum += a[e] * v[e];
                }
                q0 += W * E;
                if (q0 >= end) lane_done = true;
                else load_chunk();
            }
            const unsigned done = __ballot_sync(FULL, lane_done);
            const bool row_ready = (done & gmask) == gmask;
            const T tot = group_sum<W>(sum, FULL);
            if (row_ready && !published) {
                pubv = (bi - tot) * dinv;  // lane 0 of the group holds bi and dinv
                if (sl == 0 && i != withhold) {  // test hook: no global publication
                    st_relaxed(x + i, pubv);
                    st_release(flags + i, 1);
                }
                published = true;
            }
            if (__all_sync(FULL, published)) break;
            const unsigned pub_ballot = __ballot_sync(FULL, published);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const bool want = (pend & local & (1u << e)) != 0;
                const int g2 = want ? (upper ? i0 - c[e] : c[e] - i0) : grp;
                const T got = __shfl_sync(FULL, pubv, g2 * W);
                if (want && ((pub_ballot >> (g2 * W)) & 1u)) {
                    v[e] = got;
                    pend &= ~(1u << e);
                }
            }
            if (__any_sync(FULL, (pend & ~local) != 0)) {
                const unsigned far = pend & ~local;
#pragma unroll
                for (int e = 0; e < E; ++e)
                    if ((far & (1u << e)) && ld_acquire(flags + c[e]) != 0) {
                        v[e] = ld_relaxed(x + c[e]);
                        pend &= ~(1u << e);
                    }
                if (++waits >= sp.limit) {
                    const unsigned still = pend & ~local;
                    if (still) {
                        report(&h->status, i, kCodeTimeout);
#pragma unroll
                        for (int e = 0; e < E; ++e)
                            if (still & (1u << e)) v[e] = Marker<T>::canonical_nan();
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
}

constexpr int kMaxDevices = 64;

// Resident blocks per SM of noalloc_solve_k<T, W> at 256 threads, looked up
// once per device (0: not yet known).
template <typename T, int W>
cudaError_t blocks_per_sm(int dev, int* out) {
    static std::atomic<int> cache[kMaxDevices];
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        cudaError_t e =
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, noalloc_solve_k<T, W>, 256, 0);
        if (e != cudaSuccess) return e;
        if (v < 1) v = 1;
        cache[dev].store(v, std::memory_order_relaxed);
    }
    *out = v;
    return cudaSuccess;
}

template <typename T, int W>
cudaError_t launch_w(int n, const int* ptr, const int* idx, const void* vals, bool upper,
                     bool unit, const void* b, void* x, unsigned char* scratch, int dev,
                     int num_sms, const SpinPolicy& sp, int withhold, cudaStream_t s) {
    int per_sm = 0;
    cudaError_t e = blocks_per_sm<T, W>(dev, &per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm > 4) per_sm = 4;
    const long long tickets = ((long long)n + 32 / W - 1) / (32 / W);
    long long grid = (long long)per_sm * num_sms;
    if (grid > (tickets + 7) / 8) grid = (tickets + 7) / 8;
    if (grid < 1) grid = 1;
    noalloc_solve_k<T, W><<<(int)grid, 256, 0, s>>>(n, ptr, idx, (const T*)vals, upper, unit,
                                                   (const T*)b, (T*)x, scratch, sp, withhold);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_t(int lanes, int n, const int* ptr, const int* idx, const void* vals,
                     bool upper, bool unit, const void* b, void* x, unsigned char* scratch,
                     int dev, int num_sms, const SpinPolicy& sp, int withhold, cudaStream_t s) {
#define SPTRSV_NOALLOC(WW)                                                                  \
    return launch_w<T, WW>(n, ptr, idx, vals, upper, unit, b, x, scratch, dev, num_sms, sp, \
                           withhold, s)
    switch (lanes) {
        case 1: SPTRSV_NOALLOC(1);
        case 2: SPTRSV_NOALLOC(2);
        case 4: SPTRSV_NOALLOC(4);
        case 8: SPTRSV_NOALLOC(8);
        case 16: SPTRSV_NOALLOC(16);
        default: SPTRSV_NOALLOC(32);
    }
#undef SPTRSV_NOALLOC
}

// A positive integer from the environment, else dflt.
long long env_value(const char* name, long long dflt) {
    const char* v = getenv(name);
    if (!v || !*v) return dflt;
    char* end = nullptr;
    const long long x = strtoll(v, &end, 0);
    return (end && *end == 0 && x > 0) ? x : dflt;
}

// Device address of the scratch array, looked up once per device with that
// device current (the host-side symbol is only a stand-in, not an address).
std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

cudaError_t scratch_for_current_device(unsigned char** out, int* num_sms, int* device) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = (unsigned char*)p;
        g_num_sms[dev] = sms;
    }
    *out = g_scratch_addr[dev];
    *num_sms = g_num_sms[dev];
    *device = dev;
    return cudaSuccess;
}

}  // namespace
}  // namespace sptrsv

using namespace sptrsv;

extern "C" SPTRSV_API sptrsv_status_t sptrsv_solve_noalloc(
    int n, int nnz, const int* d_rowptr, const int* d_colidx, const void* d_vals,
    sptrsv_dtype_t dtype, sptrsv_uplo_t uplo, sptrsv_diag_t diag, const void* d_b, void* d_x,
    void* stream, int* error_row) {
    if (error_row) *error_row = -1;
    if (n < 0 || nnz < 0 || (dtype != SPTRSV_F64 && dtype != SPTRSV_F32) ||
        (uplo != SPTRSV_LOWER && uplo != SPTRSV_UPPER) ||
        (diag != SPTRSV_NON_UNIT && diag != SPTRSV_UNIT))
        return SPTRSV_ERR_INVALID_ARG;
    if (n > SPTRSV_NOALLOC_MAX_ROWS) return SPTRSV_ERR_INVALID_ARG;  // beyond the scratch array
    if (nnz > SPTRSV_MAX_SIZE) return SPTRSV_ERR_INVALID_ARG;
    if (n == 0) return SPTRSV_OK;
    if (!d_rowptr || !d_b || !d_x || (nnz > 0 && (!d_colidx || !d_vals)))
        return SPTRSV_ERR_INVALID_ARG;
    if (nnz == 0 && diag == SPTRSV_NON_UNIT) {
        if (error_row) *error_row = 0;
        return SPTRSV_ERR_ZERO_PIVOT;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* scratch = nullptr;
    int num_sms = 1, dev = 0;
    if (scratch_for_current_device(&scratch, &num_sms, &dev) != cudaSuccess)
        return SPTRSV_ERR_CUDA;
    // the bounded wait: SPTRSV_SPIN_LIMIT polls (2^24 by default), read at
    // every call; SPTRSV_DEBUG_NOALLOC_WITHHOLD = r (test hook) keeps row r
    // from being published to the other warps, so its dependents in later
    // tickets run into the limit and report SPTRSV_ERR_TIMEOUT
    const SpinPolicy sp{env_value("SPTRSV_SPIN_LIMIT", 1ll << 24), 256, 128};
    const long long wh = env_value("SPTRSV_DEBUG_NOALLOC_WITHHOLD", -1);
    const int withhold = wh >= 0 && wh < n ? (int)wh : -1;
    const bool f64 = dtype == SPTRSV_F64;
    const bool upper = uplo == SPTRSV_UPPER;
    const bool unit = diag == SPTRSV_UNIT;
    unsigned long long* status = &((Header*)scratch)->status;
    long long g = ((long long)n + 255) / 256;
    if (g > 8L * num_sms) g = 8L * num_sms;
    noalloc_clear_k<<<(int)g, 256, 0, s>>>(scratch, n);
    if (cudaGetLastError() != cudaSuccess) return SPTRSV_ERR_CUDA;
    if (launch_validate(n, nnz, d_rowptr, d_colidx, d_vals, f64, upper, unit, status,
                        num_sms * 32, s) != cudaSuccess)
        return SPTRSV_ERR_CUDA;
    double off = (double)nnz / n - 1.0;
    int lanes = 1;
    while (lanes < 32 && lanes * kChunk < off) lanes <<= 1;
    cudaError_t e = f64 ? launch_t<double>(lanes, n, d_rowptr, d_colidx, d_vals, upper, unit, d_b,
                                           d_x, scratch, dev, num_sms, sp, withhold, s)
                        : launch_t<float>(lanes, n, d_rowptr, d_colidx, d_vals, upper, unit, d_b,
                                          d_x, scratch, dev, num_sms, sp, withhold, s);
    if (e != cudaSuccess) return SPTRSV_ERR_CUDA;
    if (!error_row) return SPTRSV_OK;
    unsigned long long h = kStatusClear;
    if (cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SPTRSV_ERR_CUDA;
    if (h == kStatusClear) return SPTRSV_OK;
    *error_row = (int)(h >> 32);
    return (sptrsv_status_t)(unsigned)(h & 0xffffffffu);
}
