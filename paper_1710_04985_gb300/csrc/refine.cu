// Mixed-precision iterative refinement in one self-scheduled pass (the
// precision form: FP32 bulk solves, FP64 residuals and updates; the
// motivation is the refinement use of Sec. 1).
//
// Classical refinement alternates whole passes: solve L d0 = b in FP32,
// x1 = d0; then r1 = b - L x1 in FP64, solve L d1 = r1 in FP32, x2 = x1 + d1;
// and so on, each pass a full sweep of the dependency chain, with the host
// reading a residual norm in between.  Row i of every one of these quantities
// depends only on rows j <= i of the same or earlier passes: r^m_i needs x^m
// of row i's dependencies, d^m_i needs r^m_i and d^m of its dependencies.
// So all K+1 passes can run in one self-scheduled sweep: a row, once taken,
// computes its residual and correction for m = 0, 1, ..., K in turn, each
// step waiting (bounded) for its dependencies' values of the same step, and
// publishes d^m_i and x^{m+1}_i as it goes.  The step-m wave follows the
// step-(m-1) wave through the matrix a few rows behind instead of starting
// over after it, and no norm is read by the host until the end.
//
// Arithmetic (per row i, on the level-ordered copy, whose values are
// pre-scaled by 1/d(i) for a non-unit matrix, so a' = a / d(i)):
//   s^m  = b(i)/d(i) - x^m(i) - sum_j a'(i,j) x^m(j)      FP64 (= r^m(i)/d(i))
//   d^m  = fp32(s^m) - sum_j a'32(i,j) d^m(j)               FP32 values,
//                                                           FP32 accumulation
//   x^{m+1}(i) = x^m(i) + d^m                               FP64
// with x^0 = 0 (s^0 = b(i)/d(i), no reads) or a given initial guess.  These are
// the same operations, in the same order per row, as the staged passes of
// sptrsv_solve_refined would do with a residual r = b - A x scaled by 1/d(i).
// The residual norms max|r^m| = max |s^m| d(i) and max|x^m| of every step
// are reduced per block and combined with one atomic each at the end.
#include "internal.h"

namespace sptrsv {

template <int W>
__global__ void __launch_bounds__(512) refine_pass_k(RefineParams r) {
    constexpr int R = 32 / W;
    constexpr int E = kChunk;
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int grp = lane / W;
    const int sl = lane - grp * W;
    const unsigned gmask = group_mask<W>(lane);
    const int K = r.K;
    // running maxima of |r^m| and |x^m| over this lane's rows (lane 0 of a
    // group only), per step m <= kRefineMaxSteps
    double rmax[kRefineMaxSteps + 1], xmx[kRefineMaxSteps + 1];
#pragma unroll
    for (int m = 0; m <= kRefineMaxSteps; ++m) rmax[m] = xmx[m] = 0.0;
    int t = 0;
    if (lane == 0) t = atomicAdd(r.ticket, 1);
    t = __shfl_sync(FULL, t, 0);
    while ((long long)t * R < r.n) {
        int tn = 0;
        if (lane == 0) tn = atomicAdd(r.ticket, 1);
        const long long k = (long long)t * R + grp;
        const bool has_row = k < r.n;
        int i = 0, beg = 0, end = 0;
        double dinv = 1.0, bi = 0.0, xi = 0.0;
        if (has_row) {
            i = r.jlev[k];
            beg = r.ptr[k];
            end = r.ptr[k + 1];
            if (sl == 0) {
                if (!r.unit) dinv = r.v64[r.diag_first ? beg : end - 1];  // 1/d(i)
                bi = r.b[(long long)i * r.ldb];
                if (r.has_init) xi = r.x[(long long)i * r.ldx];
            }
        }
        // per-row step state (uniform over the row's W lanes)
        int m = 0;
        int phase = (r.has_init ? 0 : 1);  // 0: residual sweep, 1: correction sweep
        bool row_done = !has_row;
        double s = 0.0;                     // s^m, the scaled residual (lane 0)
        // per-lane sweep state
        int q0 = beg + sl;
        int c[E];
        double a64[E], v64[E];
        float a32[E], v32[E];
        unsigned live = 0, pend = 0;
        double acc64 = 0.0;
        float acc32 = 0.0f;
        bool lane_done = true;
        long long waits = 0;
        unsigned ns = 32;
        // Lanes whose entries fit one chunk keep them (columns and both value
        // types) in registers for every sweep of every step; longer rows
        // reload their chunks per sweep.
        const bool cached = q0 + W * E >= end;
        bool have = false;
        auto load_chunk = [&]() {
            if (cached && have) {  // the lane's only chunk: poll its entries again
                pend = 0;
                const long long base = (long long)m * r.n;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (!(live & (1u << e))) continue;
                    if (phase == 0) {
                        v64[e] = ld_relaxed(r.xpub + base + c[e]);
                        if (Marker<double>::pending(v64[e])) pend |= 1u << e;
                    } else {
                        v32[e] = ld_relaxed(r.dpub + base + c[e]);
                        if (Marker<float>::pending(v32[e])) pend |= 1u << e;
                    }
                }
                return;
            }
            live = pend = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int q = q0 + e * W;
                c[e] = -1;
                if (q < end) {
                    const int cc = r.idx[q];
                    if (cc != (int)k) {
                        c[e] = cc;
                        live |= 1u << e;
                        if (cached) {
                            a64[e] = r.v64[q];
                            a32[e] = r.v32[q];
                        } else if (phase == 0) {
                            a64[e] = r.v64[q];
                        } else {
                            a32[e] = r.v32[q];
                        }
                    }
                }
            }
            have = true;
            const long long base = (long long)m * r.n;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (!(live & (1u << e))) continue;
                if (phase == 0) {
                    v64[e] = ld_relaxed(r.xpub + base + c[e]);
                    if (Marker<double>::pending(v64[e])) pend |= 1u << e;
                } else {
                    v32[e] = ld_relaxed(r.dpub + base + c[e]);
                    if (Marker<float>::pending(v32[e])) pend |= 1u << e;
                }
            }
        };
        // start a sweep of the row's entries for the current (m, phase)
        auto start_sweep = [&]() {
            q0 = beg + sl;
            acc64 = 0.0;
            acc32 = 0.0f;
            if (sl == 0) {
                if (phase == 0) acc64 = bi * dinv - xi;
                else acc32 = (float)s;
            }
            lane_done = q0 >= end;
            if (!lane_done) load_chunk();
        };
        if (!row_done) {
            if (phase == 1) s = bi * dinv;  // x^0 = 0: the first residual is b itself
            if (sl == 0) {
                if (phase == 1) rmax[0] = fmax(rmax[0], fabs(bi));
                else xmx[0] = fmax(xmx[0], fabs(xi));
            }
            start_sweep();
        }
        while (true) {
            // Re-poll pending entries at every turn of the loop, not only in the
            // wait below: while other rows of the warp work through their later
            // steps the warp may not wait for a long time, and a row still in
            // an early step must not miss a value published in the meantime.
            if (!row_done && !lane_done && pend != 0) {
                const long long base = (long long)m * r.n;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (!(pend & (1u << e))) continue;
                    if (phase == 0) {
                        v64[e] = ld_relaxed(r.xpub + base + c[e]);
                        if (!Marker<double>::pending(v64[e])) pend &= ~(1u << e);
                    } else {
                        v32[e] = ld_relaxed(r.dpub + base + c[e]);
                        if (!Marker<float>::pending(v32[e])) pend &= ~(1u << e);
                    }
                }
            }
            if (!row_done && !lane_done && pend == 0) {  // fold a complete chunk in entry order
                const int hi = 32 - __clz(live);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if (e >= hi) break;
                    if (!(live & (1u << e))) continue;
                    if (phase == 0) acc64 = fma(-a64[e], v64[e], acc64);
                    else acc32 = fmaf(-a32[e], v32[e], acc32);
                }
                q0 += W * E;
                if (q0 >= end) lane_done = true;
                else load_chunk();
            }
            const unsigned done = __ballot_sync(FULL, row_done || lane_done);
            const bool ready = !row_done && (done & gmask) == gmask;
            // rows whose lanes finished a sweep: reduce, then step
            if (__any_sync(FULL, ready)) {
                const double t64 = group_sum<W>(acc64, FULL);
                const float t32 = group_sum<W>(acc32, FULL);
                if (ready) {
                    if (phase == 0) {
                        s = t64;
                        if (sl == 0 && m <= kRefineMaxSteps) {
                            const double res = r.unit ? fabs(s) : fabs(s) / dinv;
                            rmax[m] = fmax(rmax[m], res);
                        }
                        phase = 1;
                    } else {
                        const float d = t32;
                        const double xn = xi + (double)d;
                        if (sl == 0) {
                            const long long base = (long long)m * r.n;
                            st_relaxed(r.dpub + base + k, publishable(d));
                            if (m < K)
                                st_relaxed(r.xpub + base + r.n + k, publishable(xn));
                            else
                                r.x[(long long)i * r.ldx] = xn;
                            if (m + 1 <= kRefineMaxSteps) xmx[m + 1] = fmax(xmx[m + 1], fabs(xn));
                        }
                        xi = xn;
                        ++m;
                        phase = 0;
                        if (m > K) row_done = true;
                    }
                    if (!row_done) start_sweep();
                }
            }
            if (__all_sync(FULL, row_done)) break;
            if (__any_sync(FULL, !row_done && !lane_done && pend == 0)) continue;  // fold first
            // A row that just stepped may already have finished its next sweep
            // (no entries to wait for in any of its lanes): step it before
            // waiting, or a row waiting on it in this warp would wait for a
            // value that only the outer loop can produce.
            {
                const unsigned done2 = __ballot_sync(FULL, row_done || lane_done);
                if (__any_sync(FULL, !row_done && (done2 & gmask) == gmask)) continue;
            }
            if (__any_sync(FULL, pend != 0)) {
                const unsigned before = pend;
                const long long base = (long long)m * r.n;
                do {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        if (!(pend & (1u << e))) continue;
                        if (phase == 0) {
                            v64[e] = ld_relaxed(r.xpub + base + c[e]);
                            if (!Marker<double>::pending(v64[e])) pend &= ~(1u << e);
                        } else {
                            v32[e] = ld_relaxed(r.dpub + base + c[e]);
                            if (!Marker<float>::pending(v32[e])) pend &= ~(1u << e);
                        }
                    }
                    if (++waits >= r.spin.limit) {
                        if (pend) {
                            report(r.status, i, kCodeTimeout);
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                if (!(pend & (1u << e))) continue;
                                v64[e] = Marker<double>::canonical_nan();
                                v32[e] = Marker<float>::canonical_nan();
                            }
                            pend = 0;
                        }
                        waits = 0;
                        break;
                    }
                    if (__any_sync(FULL, pend != before)) break;
                    if (waits >= r.spin.hot) {
                        __nanosleep(ns);
                        ns = ns < r.spin.max_ns ? ns * 2 : r.spin.max_ns;
                    }
                } while (true);
            } else {
                waits = 0;
                ns = 32;
            }
        }
        t = __shfl_sync(FULL, tn, 0);
    }
    // block-wide maxima, then one atomic per step and quantity
    __shared__ double red[32];
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int m = 0; m <= K && m <= kRefineMaxSteps; ++m) {
        for (int which = 0; which < 2; ++which) {
            double v = which ? xmx[m] : rmax[m];
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, off));
            if (lane == 0) red[w] = v;
            __syncthreads();
            if (w == 0) {
                v = lane < nw ? red[lane] : 0.0;
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, off));
                if (lane == 0)
                    atomicMax((which ? r.xmax : r.rmax) + m,
                              (unsigned long long)__double_as_longlong(v));
            }
            __syncthreads();
        }
    }
}

// Marker fill of the step buffers (dpub: all K+1 steps; xpub: steps 1..K and,
// with an initial guess, step 0 = the guess in position order) and the ticket.
__global__ void refine_prep_k(RefineParams r) {
    const long long n = r.n;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n * (r.K + 1);
         e += stride) {
        r.dpub[e] = Marker<float>::pending_value();
        const long long m = e / n, k = e - m * n;
        r.xpub[e] = (m == 0 && r.has_init) ? r.x[(long long)r.jlev[k] * r.ldx]
                                           : Marker<double>::pending_value();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *r.ticket = 0;
}

template <int W>
static int refine_occ(int block) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, refine_pass_k<W>, block, 0) !=
        cudaSuccess)
        return 1;
    return nb > 0 ? nb : 1;
}

int refine_blocks_per_sm(int lanes, int block) {
    switch (lanes) {
        case 1: return refine_occ<1>(block);
        case 2: return refine_occ<2>(block);
        case 4: return refine_occ<4>(block);
        case 8: return refine_occ<8>(block);
        case 16: return refine_occ<16>(block);
        default: return refine_occ<32>(block);
    }
}

cudaError_t launch_refine_pass(int lanes, const RefineParams& r, int grid, int block,
                               cudaStream_t s) {
    long long want = ((long long)r.n * (r.K + 1) + 255) / 256;
    const int pg = (int)(want < 8192 ? (want > 0 ? want : 1) : 8192);
    refine_prep_k<<<pg, 256, 0, s>>>(r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    switch (lanes) {
        case 1: refine_pass_k<1><<<grid, block, 0, s>>>(r); break;
        case 2: refine_pass_k<2><<<grid, block, 0, s>>>(r); break;
        case 4: refine_pass_k<4><<<grid, block, 0, s>>>(r); break;
        case 8: refine_pass_k<8><<<grid, block, 0, s>>>(r); break;
        case 16: refine_pass_k<16><<<grid, block, 0, s>>>(r); break;
        case 32: refine_pass_k<32><<<grid, block, 0, s>>>(r); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace sptrsv
