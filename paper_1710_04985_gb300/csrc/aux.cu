// Kernels around the solves: the sparse gradient on the matrix pattern, and
// the FP64 steps of mixed-precision iterative refinement (residual, update,
// conversions).  All are single passes over HBM with no dependencies.
#include "internal.h"

namespace sptrsv {

__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* where, double v) {
    // Non-negative doubles (and NaN, which then wins) order like their bits.
    atomicMax(where, (unsigned long long)__double_as_longlong(v));
}

// Block-wide max of a non-negative value, then one atomic per block.
__device__ __forceinline__ void block_max_to(unsigned long long* where, double v) {
    __shared__ double wmax[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wmax[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (lane == 0) atomic_max_nonneg(where, v);
    }
}

// Block-wide max of the bits of non-negative doubles (NaN, whose bits are
// larger than infinity's, wins), then one atomic per block: integer
// operations only, no FP64 instruction.
__device__ __forceinline__ void block_max_bits_to(unsigned long long* where,
                                                  unsigned long long v) {
    __shared__ unsigned long long wmax[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o > v ? o : v;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wmax[w] = v;
    __syncthreads();
    if (w == 0) {
        v = lane < (int)(blockDim.x >> 5) ? wmax[lane] : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, off);
            v = o > v ? o : v;
        }
        if (lane == 0 && v) atomicMax(where, v);
    }
}

__device__ __forceinline__ unsigned long long abs_bits(double v) {
    return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffull;
}

// ------------------------------------------------------------ gradient
// g[q] = - sum_c y[i][c] x[j][c] for stored entry q = (i, j); zero on the
// diagonal of a unit-diagonal matrix (it is not a parameter).
template <typename T, int W>
__global__ void grad_vals_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                            int unit, const T* __restrict__ y, long long ldy,
                            const T* __restrict__ x, long long ldx, int k, T* __restrict__ g) {
    const long long groups = (long long)gridDim.x * blockDim.x / W;
    const int sl = threadIdx.x % W;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / W; i < n; i += groups) {
        const int beg = ptr[i], end = ptr[i + 1];
        if (k == 1) {
            const T yi = y[i * ldy];
            for (int q = beg + sl; q < end; q += W) {
                const int j = idx[q];
                g[q] = (unit && j == i) ? T(0) : -(yi * x[(long long)j * ldx]);
            }
        } else {
            for (int q = beg + sl; q < end; q += W) {
                const int j = idx[q];
                T s = T(0);
                if (!(unit && j == i))
                    for (int c = 0; c < k; ++c) s += y[i * ldy + c] * x[(long long)j * ldx + c];
                g[q] = -s;
            }
        }
    }
}

template <typename T>
static cudaError_t grad_t(int lanes, int n, const int* ptr, const int* idx, bool unit,
                          const void* y, long long ldy, const void* x, long long ldx, int k,
                          void* g, cudaStream_t s, int grid) {
    long long want = ((long long)n * lanes + 255) / 256;
    int gg = (int)(want < grid ? want : grid);
    if (gg < 1) gg = 1;
#define SPTRSV_GRAD(W)                                                                         \
    grad_vals_k<T, W><<<gg, 256, 0, s>>>(n, ptr, idx, unit, (const T*)y, ldy, (const T*)x, ldx, \
                                         k, (T*)g)
    switch (lanes) {
        case 1: SPTRSV_GRAD(1); break;
        case 2: SPTRSV_GRAD(2); break;
        case 4: SPTRSV_GRAD(4); break;
        case 8: SPTRSV_GRAD(8); break;
        case 16: SPTRSV_GRAD(16); break;
        case 32: SPTRSV_GRAD(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef SPTRSV_GRAD
    return cudaGetLastError();
}

cudaError_t launch_grad_vals(bool f64, int lanes, int n, const int* ptr, const int* idx, bool unit,
                             const void* y, long long ldy, const void* x, long long ldx, int k,
                             void* g, cudaStream_t s, int grid) {
    if (n == 0) return cudaSuccess;
    return f64 ? grad_t<double>(lanes, n, ptr, idx, unit, y, ldy, x, ldx, k, g, s, grid)
               : grad_t<float>(lanes, n, ptr, idx, unit, y, ldy, x, ldx, k, g, s, grid);
}

// ------------------------------------------------------------ residual (FP64)
// On GB300 an FP64 warp instruction holds its sub-partition's FP64 unit for
// ~76 cycles whatever its active lanes, and this pass is bound by that unit:
// the width W is chosen so that lanes stay busy (about four entries per lane,
// residual_lanes), the maxima are integer maxima of the bits of |v|, and the
// sum of |a_ij| is formed only when the norm is asked for.
template <int W>
__global__ void residual_k(int n, const int* __restrict__ ptr, const int* __restrict__ idx,
                           const double* __restrict__ vals, int unit, int k,
                           const double* __restrict__ b, long long ldb,
                           const double* __restrict__ x, long long ldx, double* r, long long ldr,
                           float* r32, unsigned long long* stats, int want_norm) {
    const long long groups = (long long)gridDim.x * blockDim.x / W;
    const int lane = threadIdx.x & 31;
    const int sl = lane % W;
    const unsigned gmask = group_mask<W>(lane);
    unsigned long long rmax = 0, amax = 0, xmax = 0;  // bits of non-negative doubles
    // Every lane of a block runs the same number of iterations so that the
    // block-wide reduction below is reached by all of them.
    const long long first = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / W;
    const long long base0 = ((long long)blockIdx.x * blockDim.x) / W;
    for (long long i0 = base0; i0 < n; i0 += groups) {
        const long long i = first - base0 + i0;
        if (i < n) {
            const int beg = ptr[i], end = ptr[i + 1];
            for (int c = 0; c < k; ++c) {
                double s = 0.0, a_abs = 0.0;
                for (int q = beg + sl; q < end; q += W) {
                    const int j = idx[q];
                    if (unit && j == i) continue;  // a unit diagonal is added below
                    const double a = vals[q];
                    s += a * x[(long long)j * ldx + c];
                    if (c == 0 && want_norm) a_abs += fabs(a);  // FP64 adds only when asked
                }
                s = group_sum<W>(s, gmask);
                if (c == 0 && want_norm) a_abs = group_sum<W>(a_abs, gmask);
                if (unit) {  // the diagonal is 1, stored or not
                    s += x[i * ldx + c];
                    if (c == 0 && want_norm) a_abs += 1.0;
                }
                if (sl == 0) {
                    const double rr = b[i * ldb + c] - s;
                    if (r) r[i * ldr + c] = rr;
                    if (r32) r32[i * k + c] = (float)rr;
                    const unsigned long long rb = abs_bits(rr), xb = abs_bits(x[i * ldx + c]);
                    rmax = rb > rmax ? rb : rmax;
                    xmax = xb > xmax ? xb : xmax;
                    if (c == 0 && want_norm) {
                        const unsigned long long ab = abs_bits(a_abs);
                        amax = ab > amax ? ab : amax;
                    }
                }
            }
        }
    }
    if (stats) {
        block_max_bits_to(stats, rmax);
        __syncthreads();
        block_max_bits_to(stats + 2, xmax);
        if (want_norm) {
            __syncthreads();
            block_max_bits_to(stats + 1, amax);
        }
    }
}

// Width of the residual pass: about four stored entries per lane (a power of
// two in 1..32), from the average row length.
int residual_lanes(int n, long long nnz) {
    const double per_row = n > 0 ? (double)nnz / n : 1.0;
    int w = 1;
    while (w < 32 && 4.0 * (2 * w) <= per_row) w *= 2;
    return w;
}

cudaError_t launch_residual(int n, long long nnz, const int* ptr, const int* idx,
                            const double* vals, bool unit, int k, const double* b, long long ldb,
                            const double* x, long long ldx, double* r, long long ldr, float* r32,
                            unsigned long long* stats, bool want_norm, int grid, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int lanes = residual_lanes(n, nnz);
    long long want = ((long long)n * lanes + 255) / 256;
    int g = (int)(want < grid ? want : grid);
    if (g < 1) g = 1;
#define SPTRSV_RES(W)                                                                          \
    residual_k<W><<<g, 256, 0, s>>>(n, ptr, idx, vals, unit, k, b, ldb, x, ldx, r, ldr, r32, \
                                    stats, want_norm)
    switch (lanes) {
        case 1: SPTRSV_RES(1); break;
        case 2: SPTRSV_RES(2); break;
        case 4: SPTRSV_RES(4); break;
        case 8: SPTRSV_RES(8); break;
        case 16: SPTRSV_RES(16); break;
        case 32: SPTRSV_RES(32); break;
        default: return cudaErrorInvalidValue;
    }
#undef SPTRSV_RES
    return cudaGetLastError();
}

// ------------------------------------------------------------ update / convert
__global__ void update_k(int n, int k, double* x, long long ldx, const float* __restrict__ d,
                         int first, unsigned long long* xmax) {
    const long long total = (long long)n * k;
    double m = 0.0;
    for (long long e0 = (long long)blockIdx.x * blockDim.x; e0 < total;
         e0 += (long long)gridDim.x * blockDim.x) {
        const long long e = e0 + threadIdx.x;
        if (e < total) {
            const long long r = e / k, c = e - r * k;
            double* xp = x + r * ldx + c;
            const double v = first ? (double)d[e] : *xp + (double)d[e];
            *xp = v;
            m = fmax(m, fabs(v));
        }
    }
    if (xmax) block_max_to(xmax, m);
}

cudaError_t launch_update(int n, int k, double* x, long long ldx, const float* d, bool first,
                          unsigned long long* xmax, int grid, cudaStream_t s) {
    const long long total = (long long)n * k;
    if (total == 0) return cudaSuccess;
    long long want = (total + 255) / 256;
    int g = (int)(want < grid ? want : grid);
    update_k<<<g, 256, 0, s>>>(n, k, x, ldx, d, first, xmax);
    return cudaGetLastError();
}

__global__ void to_f32_k(int n, int k, const double* __restrict__ in, long long ldin,
                         float* __restrict__ out, unsigned long long* amax) {
    const long long total = (long long)n * k;
    double m = 0.0;
    for (long long e0 = (long long)blockIdx.x * blockDim.x; e0 < total;
         e0 += (long long)gridDim.x * blockDim.x) {
        const long long e = e0 + threadIdx.x;
        if (e < total) {
            const long long r = e / k, c = e - r * k;
            const double v = in[r * ldin + c];
            out[e] = (float)v;
            m = fmax(m, fabs(v));
        }
    }
    if (amax) block_max_to(amax, m);
}

cudaError_t launch_to_f32(int n, int k, const double* in, long long ldin, float* out,
                          unsigned long long* amax, int grid, cudaStream_t s) {
    const long long total = (long long)n * k;
    if (total == 0) return cudaSuccess;
    long long want = (total + 255) / 256;
    int g = (int)(want < grid ? want : grid);
    to_f32_k<<<g, 256, 0, s>>>(n, k, in, ldin, out, amax);
    return cudaGetLastError();
}

}  // namespace sptrsv
