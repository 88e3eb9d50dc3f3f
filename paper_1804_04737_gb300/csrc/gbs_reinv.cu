// FP64 reinversion for the FP32-tableau mode.
//
// The FP32 tableau carries rounding error that grows with the pivots.  Every
// reinv_k pivots and at termination the library recomputes, in FP64 and from
// the original data, the parts of the tableau that decide the next pivots and
// certify the answer:
//   x_B = B^-1 rhs   (the rhs column),
//   y   = duals, and the objective row  z_j = (A'y)_j - c_j, slacks z = y,
//   z*  = c_B' x_B,
// for the current basis B (the columns of [A I] that are basic).  With s
// structural basic variables S and the m - s rows L whose slack is basic, and
// R the s rows whose slack is not, B is block triangular:
//   B = [[A_RS, 0], [A_LS, I]]  =>  x_S = A_RS^-1 b_R,  x_L = b_L - A_LS x_S,
//                                   y_R = A_RS^-T c_S,  y_L = 0,
// so the work is one s x s Gauss-Jordan elimination (partial pivoting, on
// [A_RS | b_R | I]) and matrix-vector products; the body B^-1 A of the tableau
// stays in FP32.  The refreshed rhs column and objective row are rounded into
// the FP32 tableau, and the FP64 values are the reported solution.  The check
// reports the smallest objective-row entry and the smallest rhs so the host
// can test optimality and feasibility in FP64.
//
// Sign conventions follow the tableau: for the dual form the data enter as
// (-A, -b, -c) (the objective row holds c and the rhs -b initially).

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "gbs_device.cuh"
#include "gbs_internal.h"

namespace gbs {
namespace {

using namespace dev;

// Index lists of the basis (one CTA): Lflag[l] = slack of row l is basic;
// S = structural basic variables (in row order), R = rows whose slack is not
// basic (ascending); posS[j] = k with S[k] = j or -1; posR[l] = r with R[r] = l
// or -1; counts[0] = |S|, counts[1] = |R|.
__device__ __forceinline__ void lists_cta(const int *__restrict__ basis, int m, int n, int *Lflag,
                                          int *S, int *R, int *posS, int *posR, int *counts) {
    __shared__ int scanS[1024], scanR[1024];
    const int tid = threadIdx.x, B = blockDim.x;
    for (int l = tid; l < m; l += B) Lflag[l] = 0;
    for (int j = tid; j < n; j += B) posS[j] = -1;
    __syncthreads();
    for (int i = tid; i < m; i += B) {
        const int v = basis[i];
        if (v >= n) Lflag[v - n] = 1;
    }
    __syncthreads();
    const int chunk = (m + B - 1) / B;
    const int i0 = min(m, tid * chunk), i1 = min(m, i0 + chunk);
    int cS = 0, cR = 0;
    for (int i = i0; i < i1; ++i) {
        cS += basis[i] < n;
        cR += Lflag[i] == 0;
    }
    scanS[tid] = cS;
    scanR[tid] = cR;
    __syncthreads();
    for (int o = 1; o < B; o <<= 1) {  // inclusive Hillis-Steele scan
        const int a = tid >= o ? scanS[tid - o] : 0;
        const int b = tid >= o ? scanR[tid - o] : 0;
        __syncthreads();
        scanS[tid] += a;
        scanR[tid] += b;
        __syncthreads();
    }
    int kS = scanS[tid] - cS, kR = scanR[tid] - cR;
    for (int i = i0; i < i1; ++i) {
        const int v = basis[i];
        if (v < n) {
            S[kS] = v;
            posS[v] = kS;
            ++kS;
        }
        if (Lflag[i] == 0) {
            R[kR] = i;
            posR[i] = kR;
            ++kR;
        } else {
            posR[i] = -1;
        }
    }
    if (tid == B - 1) {
        counts[0] = scanS[tid];
        counts[1] = scanR[tid];
    }
}

__global__ void __launch_bounds__(1024) reinv_lists_kernel(const int *__restrict__ basis, int m,
                                                           int n, int *Lflag, int *S, int *R,
                                                           int *posS, int *posR, int *counts) {
    lists_cta(basis, m, n, Lflag, S, R, posS, posR, counts);
}

// The lists of many LPs, one CTA each.
__global__ void __launch_bounds__(1024) reinv_lists_batch_kernel(const ReinvItem *__restrict__ it) {
    const ReinvItem &r = it[blockIdx.x];
    lists_cta(r.basis, r.m, r.n, r.Lflag, r.S, r.R, r.posS, r.posR, r.counts);
}

// W = [A_RS | b_R | I_s] (signed data), s rows, pitch Wp >= 2s + 1.
__global__ void reinv_gather_kernel(const double *__restrict__ A, const double *__restrict__ b,
                                    double sg, int n, const int *__restrict__ S,
                                    const int *__restrict__ R, int s, double *__restrict__ W,
                                    long long Wp) {
    const long long total = (long long)s * Wp;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += stride) {
        const int r = (int)(k / Wp);
        const int j = (int)(k - (long long)r * Wp);
        double v = 0.0;
        if (j < s) v = sg * A[(long long)R[r] * n + S[j]];
        else if (j == s) v = sg * b[R[r]];
        else if (j - s - 1 == r) v = 1.0;
        W[k] = v;
    }
}

// Gauss-Jordan elimination with partial pivoting on W (s x ncols, pitch Wp),
// one persistent grid, column strips of width `strip` per CTA.  Step k: every
// CTA picks the unused row with the largest |W[i][k]| (ties: smallest row) and
// stages column k; after a grid barrier each CTA eliminates column k from its
// strip (pivot row divided by the pivot, the others one fma per element); a
// second barrier ends the step.  pivrow[k] receives the row of step k;
// *singular is set when a column has no nonzero unused entry.
__global__ void __launch_bounds__(1024) gj_kernel(double *__restrict__ W, long long Wp, int s,
                                                  int ncols, int strip, int *pivrow,
                                                  int *singular, unsigned *bar, int *err,
                                                  long long spin_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *colk = reinterpret_cast<double *>(smem_raw);
    double *prow = colk + s;
    unsigned *used = reinterpret_cast<unsigned *>(prow + strip);
    __shared__ Cand rbuf[32];
    __shared__ int s_flag;
    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
    const int c0 = g * strip, c1 = min(ncols, c0 + strip), w = c1 - c0;
    for (int k = tid; k < (s + 31) / 32; k += B) used[k] = 0u;
    __syncthreads();
    for (int k = 0; k < s; ++k) {
        Cand c = cand_empty();
        for (int i = tid; i < s; i += B) {
            const double x = __ldcg(W + (long long)i * Wp + k);
            colk[i] = x;
            if (!((used[i >> 5] >> (i & 31)) & 1u)) {
                const unsigned long long ak =
                    ((unsigned long long)__double_as_longlong(x) & ~kSign) | kSign;
                cand_take(c, ~ak, i, i);
            }
        }
        c = block_min_c(c, rbuf);
        const int p = c.idx;
        if (p < 0 || (((unsigned long long)__double_as_longlong(colk[p])) & ~kSign) == 0ull) {
            if (g == 0 && tid == 0) *singular = 1;
            break;  // every CTA sees the same column
        }
        if (tid == 0) used[p >> 5] |= 1u << (p & 31);
        if (!grid_sync(bar, err, G, spin_limit, &s_flag)) break;
        const double piv = colk[p];
        for (int j = c0 + tid; j < c1; j += B) prow[j - c0] = __ldcg(W + (long long)p * Wp + j) / piv;
        __syncthreads();
        if (w > 0) {
            for (long long e = tid; e < (long long)s * w; e += B) {
                const int i = (int)(e / w);
                const int j = c0 + (int)(e - (long long)i * w);
                double *q = W + (long long)i * Wp + j;
                *q = i == p ? prow[j - c0] : fma(-colk[i], prow[j - c0], *q);
            }
        }
        if (g == 0 && tid == 0) pivrow[k] = p;
        if (!grid_sync(bar, err, G, spin_limit, &s_flag)) break;
    }
}

// x_S[k] = W[pivrow[k]][s];  y_R[r] = sum_k (A_RS^-1)[k][r] c_S[k], where row
// pivrow[k] of the right block holds row k of A_RS^-1.
__global__ void reinv_solve_kernel(const double *__restrict__ W, long long Wp, int s,
                                   const int *__restrict__ pivrow, const int *__restrict__ S,
                                   const double *__restrict__ c, double sg, double *xS,
                                   double *yR, const int *__restrict__ singular) {
    if (*singular) return;  // pivrow holds only the steps made; the host reports the LP numerical
    const int stride = gridDim.x * blockDim.x;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < s; r += stride) {
        xS[r] = W[(long long)pivrow[r] * Wp + s];
        double acc = 0.0;
        for (int k = 0; k < s; ++k)
            acc = fma(W[(long long)pivrow[k] * Wp + s + 1 + r], sg * c[S[k]], acc);
        yR[r] = acc;
    }
}

// Objective row in FP64: z_j = sum_r A[R[r]][j] y_R[r] - c_j for structural
// j (0 when basic), z_{n+l} = y_l for slacks (0 when basic).
__global__ void reinv_objrow_kernel(const double *__restrict__ A, const double *__restrict__ c,
                                    double sg, int m, int n, const int *__restrict__ R,
                                    const int *__restrict__ posS, const int *__restrict__ posR,
                                    int s, const double *__restrict__ yR, double *zrow) {
    const int stride = gridDim.x * blockDim.x;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n + m; j += stride) {
        double z = 0.0;
        if (j < n) {
            if (posS[j] < 0) {
                double acc = 0.0;
                for (int r = 0; r < s; ++r) acc = fma(sg * A[(long long)R[r] * n + j], yR[r], acc);
                z = acc - sg * c[j];
            }
        } else {
            const int r = posR[j - n];
            z = r >= 0 ? yR[r] : 0.0;
        }
        zrow[j] = z;
    }
}

// rhs of every tableau row: x_S for structural basics, b_l - A_lS x_S for the
// slack basic of row l.
__global__ void reinv_rhs_kernel(const double *__restrict__ A, const double *__restrict__ b,
                                 double sg, int m, int n, const int *__restrict__ basis,
                                 const int *__restrict__ S, const int *__restrict__ posS, int s,
                                 const double *__restrict__ xS, double *rhs) {
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int v = basis[i];
        double r;
        if (v < n) {
            r = xS[posS[v]];
        } else {
            const int l = v - n;
            double acc = sg * b[l];
            for (int k = 0; k < s; ++k) acc = fma(-(sg * A[(long long)l * n + S[k]]), xS[k], acc);
            r = acc;
        }
        rhs[i] = r;
    }
}

// One CTA: objective value z* = sum_k c_S[k] x_S[k] (fixed-order tree), the
// solution vectors, the refreshed FP32 rhs column and objective row, and the
// check minima.
template <typename T>
__global__ void __launch_bounds__(1024) reinv_apply_kernel(
    const double *__restrict__ c, double sg, int m, int n, const int *__restrict__ S,
    const int *__restrict__ posS, int s, const double *__restrict__ xS,
    const double *__restrict__ zrow, const double *__restrict__ rhs, T *Tab, long long P,
    double *x, double *y, double *obj, ReinvCheck *chk) {
    __shared__ double part[1024];
    const int tid = threadIdx.x, B = blockDim.x;
    const int N = n + m + 1;
    double acc = 0.0;
    for (int k = tid; k < s; k += B) acc = fma(sg * c[S[k]], xS[k], acc);
    part[tid] = acc;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (tid < o && tid + o < B) part[tid] += part[tid + o];
        __syncthreads();
    }
    const double z = part[0];
    unsigned long long zmin = ~0ull, rmin = ~0ull;
    for (int j = tid; j < n + m; j += B) {
        const double v = zrow[j];
        Tab[(long long)m * P + j] = (T)v;
        const unsigned long long k = okey(v);
        zmin = k < zmin ? k : zmin;
        if (j < n) x[j] = posS[j] >= 0 ? xS[posS[j]] : 0.0;
        else y[j - n] = v;
    }
    for (int i = tid; i < m; i += B) {
        const double v = rhs[i];
        Tab[(long long)i * P + (N - 1)] = (T)v;
        const unsigned long long k = okey(v);
        rmin = k < rmin ? k : rmin;
    }
    if (tid == 0) {
        Tab[(long long)m * P + (N - 1)] = (T)z;
        *obj = sg > 0 ? z : -z;
    }
    atomicMin(&chk->zmin_key, zmin);
    atomicMin(&chk->rhsmin_key, rmin);
}


// The whole reinversion of one LP in one CTA of 1024 threads (LPs with at
// most kReinvCtaMax structural basics, lists already made): W, Gauss-Jordan,
// x_S and y_R, objective row, rhs, and the apply step, each element with the
// operations and in the order of the multi-CTA kernels above (the objective
// sum uses the same 1024-thread tree), so the results are the same bits.
template <typename T>
__global__ void __launch_bounds__(1024) reinv_cta_kernel(const ReinvItem *__restrict__ items) {
    __shared__ double colk[kReinvCtaMax], prow[2 * kReinvCtaMax + 1], part[1024];
    __shared__ unsigned used[(kReinvCtaMax + 31) / 32];
    __shared__ int piv_row[kReinvCtaMax];
    __shared__ Cand rbuf[32];
    __shared__ int s_sing;
    const ReinvItem &it = items[blockIdx.x];
    const int tid = threadIdx.x, B = blockDim.x;
    const int m = it.m, n = it.n, ns = it.ns, ncols = 2 * ns + 1;
    const double sg = it.sense == 0 ? 1.0 : -1.0;
    const double *A = it.A, *b = it.b, *c = it.c;
    const int *S = it.S, *R = it.R, *posS = it.posS, *posR = it.posR;
    const long long Wp = it.Wp;
    double *W = it.W;
    if (tid == 0) {
        s_sing = 0;
        it.chk->zmin_key = ~0ull;
        it.chk->rhsmin_key = ~0ull;
        it.chk->singular = 0;
    }
    for (long long k = tid; k < (long long)ns * Wp; k += B) {
        const int r = (int)(k / Wp);
        const int j = (int)(k - (long long)r * Wp);
        double v = 0.0;
        if (j < ns) v = sg * A[(long long)R[r] * n + S[j]];
        else if (j == ns) v = sg * b[R[r]];
        else if (j - ns - 1 == r) v = 1.0;
        W[k] = v;
    }
    for (int k = tid; k < (ns + 31) / 32; k += B) used[k] = 0u;
    __syncthreads();
    for (int k = 0; k < ns; ++k) {
        Cand cd = cand_empty();
        for (int i = tid; i < ns; i += B) {
            const double x = W[(long long)i * Wp + k];
            colk[i] = x;
            if (!((used[i >> 5] >> (i & 31)) & 1u)) {
                const unsigned long long ak =
                    ((unsigned long long)__double_as_longlong(x) & ~kSign) | kSign;
                cand_take(cd, ~ak, i, i);
            }
        }
        cd = block_min_c(cd, rbuf);
        const int p = cd.idx;
        if (p < 0 || (((unsigned long long)__double_as_longlong(colk[p])) & ~kSign) == 0ull) {
            if (tid == 0) s_sing = 1;
            break;  // every thread sees the same column
        }
        const double piv = colk[p];
        for (int j = tid; j < ncols; j += B) prow[j] = W[(long long)p * Wp + j] / piv;
        if (tid == 0) {
            used[p >> 5] |= 1u << (p & 31);
            piv_row[k] = p;
        }
        __syncthreads();
        for (long long e = tid; e < (long long)ns * ncols; e += B) {
            const int i = (int)(e / ncols);
            const int j = (int)(e - (long long)i * ncols);
            double *q = W + (long long)i * Wp + j;
            *q = i == p ? prow[j] : fma(-colk[i], prow[j], *q);
        }
        __syncthreads();
    }
    __syncthreads();
    if (s_sing) {  // the host reports the LP numerical; nothing else is read
        if (tid == 0) it.chk->singular = 1;
        return;
    }
    double *xS = it.xS, *yR = it.yR, *zrow = it.zrow, *rhs = it.rhs;
    for (int r = tid; r < ns; r += B) {
        xS[r] = W[(long long)piv_row[r] * Wp + ns];
        double acc = 0.0;
        for (int k = 0; k < ns; ++k)
            acc = fma(W[(long long)piv_row[k] * Wp + ns + 1 + r], sg * c[S[k]], acc);
        yR[r] = acc;
    }
    __syncthreads();
    for (int j = tid; j < n + m; j += B) {
        double z = 0.0;
        if (j < n) {
            if (posS[j] < 0) {
                double acc = 0.0;
                for (int r = 0; r < ns; ++r) acc = fma(sg * A[(long long)R[r] * n + j], yR[r], acc);
                z = acc - sg * c[j];
            }
        } else {
            const int r = posR[j - n];
            z = r >= 0 ? yR[r] : 0.0;
        }
        zrow[j] = z;
    }
    for (int i = tid; i < m; i += B) {
        const int v = it.basis[i];
        double r;
        if (v < n) {
            r = xS[posS[v]];
        } else {
            const int l = v - n;
            double acc = sg * b[l];
            for (int k = 0; k < ns; ++k) acc = fma(-(sg * A[(long long)l * n + S[k]]), xS[k], acc);
            r = acc;
        }
        rhs[i] = r;
    }
    __syncthreads();
    // the apply step (reinv_apply_kernel with 1024 threads)
    T *Tab = reinterpret_cast<T *>(it.T);
    const long long P = it.P;
    const int N = n + m + 1;
    double acc = 0.0;
    for (int k = tid; k < ns; k += B) acc = fma(sg * c[S[k]], xS[k], acc);
    part[tid] = acc;
    __syncthreads();
    for (int o = 512; o > 0; o >>= 1) {
        if (tid < o && tid + o < B) part[tid] += part[tid + o];
        __syncthreads();
    }
    const double z = part[0];
    unsigned long long zmin = ~0ull, rmin = ~0ull;
    for (int j = tid; j < n + m; j += B) {
        const double v = zrow[j];
        Tab[(long long)m * P + j] = (T)v;
        const unsigned long long k = okey(v);
        zmin = k < zmin ? k : zmin;
        if (j < n) it.x[j] = posS[j] >= 0 ? xS[posS[j]] : 0.0;
        else it.y[j - n] = v;
    }
    for (int i = tid; i < m; i += B) {
        const double v = rhs[i];
        Tab[(long long)i * P + (N - 1)] = (T)v;
        const unsigned long long k = okey(v);
        rmin = k < rmin ? k : rmin;
    }
    if (tid == 0) {
        Tab[(long long)m * P + (N - 1)] = (T)z;
        *it.obj = sg > 0 ? z : -z;
    }
    atomicMin(&it.chk->zmin_key, zmin);
    atomicMin(&it.chk->rhsmin_key, rmin);
}

int grid_of(long long work) {
    long long g = (work + 255) / 256;
    return (int)(g < 1 ? 1 : (g > 2432 ? 2432 : g));
}

}  // namespace

cudaError_t launch_reinv_lists_batch(const ReinvItem *d_items, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    reinv_lists_batch_kernel<<<count, 1024, 0, s>>>(d_items);
    return cudaGetLastError();
}

cudaError_t launch_reinv_solve_batch(int prec, const ReinvItem *d_items, int count, cudaStream_t s) {
    if (count <= 0) return cudaSuccess;
    if (prec == PREC_FP64) reinv_cta_kernel<double><<<count, 1024, 0, s>>>(d_items);
    else reinv_cta_kernel<float><<<count, 1024, 0, s>>>(d_items);
    return cudaGetLastError();
}

cudaError_t launch_reinv_lists(const int *basis, int m, int n, const ReinvBufs &rb,
                               cudaStream_t s) {
    reinv_lists_kernel<<<1, 1024, 0, s>>>(basis, m, n, rb.Lflag, rb.S, rb.R, rb.posS, rb.posR,
                                          rb.counts);
    return cudaGetLastError();
}

cudaError_t launch_reinv_solve(int prec, const double *A, const double *b, const double *c,
                               int sense, int m, int n, const int *basis, const ReinvBufs &rb,
                               int ns, void *T, long long P, double *x, double *y, double *obj,
                               int sms, long long spin_limit, cudaStream_t s) {
    const double sg = sense == 0 ? 1.0 : -1.0;
    cudaError_t e = cudaMemsetAsync(rb.chk, 0xff, sizeof(ReinvCheck), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&rb.chk->singular, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (ns > 0) {
        const long long Wp = rb.Wp;
        reinv_gather_kernel<<<grid_of((long long)ns * Wp), 256, 0, s>>>(A, b, sg, n, rb.S, rb.R,
                                                                         ns, rb.W, Wp);
        const int ncols = 2 * ns + 1;
        int G = ncols / 64 > 0 ? ncols / 64 : 1;  // strips of >= 64 columns
        if (G > sms) G = sms;
        int strip = (ncols + G - 1) / G;
        G = (ncols + strip - 1) / strip;
        const size_t smem = sizeof(double) * ((size_t)ns + strip) + 4 * (((size_t)ns + 31) / 32);
        const void *fn = (const void *)gj_kernel;
        if (smem > 0) {  // static shared memory counts against the 48 KB default too
            e = allow_dyn_smem(fn);
            if (e != cudaSuccess) return e;
        }
        e = cudaMemsetAsync(rb.bar, 0, 128 * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        double *W = rb.W;
        int *pivrow = rb.pivrow;
        int *singular = &rb.chk->singular;
        unsigned *bar = rb.bar;
        int *err = reinterpret_cast<int *>(rb.bar + 96);
        int threads = 256;
        void *args[] = {&W, (void *)&Wp, &ns, (void *)&ncols, &strip, &pivrow, &singular, &bar,
                        &err, &spin_limit};
        e = cudaLaunchCooperativeKernel(fn, dim3(G), dim3(threads), args, smem, s);
        if (e != cudaSuccess) return e;
        reinv_solve_kernel<<<grid_of(ns), 256, 0, s>>>(W, Wp, ns, pivrow, rb.S, c, sg, rb.xS,
                                                       rb.yR, singular);
    }
    reinv_objrow_kernel<<<grid_of(n + m), 256, 0, s>>>(A, c, sg, m, n, rb.R, rb.posS, rb.posR, ns,
                                                       rb.yR, rb.zrow);
    reinv_rhs_kernel<<<grid_of(m), 256, 0, s>>>(A, b, sg, m, n, basis, rb.S, rb.posS, ns, rb.xS,
                                                rb.rhs);
    if (prec == PREC_FP64)
        reinv_apply_kernel<double><<<1, 1024, 0, s>>>(c, sg, m, n, rb.S, rb.posS, ns, rb.xS,
                                                      rb.zrow, rb.rhs, (double *)T, P, x, y, obj,
                                                      rb.chk);
    else
        reinv_apply_kernel<float><<<1, 1024, 0, s>>>(c, sg, m, n, rb.S, rb.posS, ns, rb.xS,
                                                     rb.zrow, rb.rhs, (float *)T, P, x, y, obj,
                                                     rb.chk);
    return cudaGetLastError();
}

namespace {
template <typename X>
cudaError_t grow_dev(X **p, size_t *cap, size_t need) {
    if (need <= *cap) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(p, need * sizeof(X));
    if (e == cudaSuccess) *cap = need;
    return e;
}
}  // namespace

BatchReinv::~BatchReinv() {
    if (d_int) cudaFree(d_int);
    if (d_counts) cudaFree(d_counts);
    if (h_counts) cudaFreeHost(h_counts);
    if (d_dbl) cudaFree(d_dbl);
    if (d_W) cudaFree(d_W);
    if (d_items) cudaFree(d_items);
    if (h_items) cudaFreeHost(h_items);
    if (d_chk) cudaFree(d_chk);
    if (h_chk) cudaFreeHost(h_chk);
}

cudaError_t reinvert_many(int prec, const ReinvJob *jobs, int count, BatchReinv &ws,
                          ReinvPool &rp, int sms, long long spin_limit, cudaStream_t s, int *bad) {
    *bad = -1;
    if (count <= 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    if ((size_t)count > ws.cap_n) {
        if (ws.d_counts) cudaFree(ws.d_counts);
        if (ws.h_counts) cudaFreeHost(ws.h_counts);
        if (ws.d_items) cudaFree(ws.d_items);
        if (ws.h_items) cudaFreeHost(ws.h_items);
        if (ws.d_chk) cudaFree(ws.d_chk);
        if (ws.h_chk) cudaFreeHost(ws.h_chk);
        ws.d_counts = ws.h_counts = nullptr;
        ws.d_items = ws.h_items = nullptr;
        ws.d_chk = ws.h_chk = nullptr;
        ws.cap_n = 0;
        e = cudaMalloc(&ws.d_counts, 2 * (size_t)count * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&ws.h_counts, 2 * (size_t)count * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&ws.d_items, (size_t)count * sizeof(ReinvItem));
        if (e == cudaSuccess) e = cudaMallocHost(&ws.h_items, (size_t)count * sizeof(ReinvItem));
        if (e == cudaSuccess) e = cudaMalloc(&ws.d_chk, (size_t)count * sizeof(ReinvCheck));
        if (e == cudaSuccess) e = cudaMallocHost(&ws.h_chk, (size_t)count * sizeof(ReinvCheck));
        if (e != cudaSuccess) return e;
        ws.cap_n = count;
    }
    // slices: ints Lflag (m), S (n), R (m), posS (n), posR (m); doubles xS, yR
    // (min(m, n) + 1 each), zrow (n + m), rhs (m)
    size_t ni = 0, nd = 0;
    for (int k = 0; k < count; ++k) {
        const size_t m = jobs[k].m, n = jobs[k].n, mn = std::min(m, n) + 1;
        ni += (3 * m + 2 * n + 63) / 64 * 64;
        nd += (2 * mn + n + 2 * m + 31) / 32 * 32;
    }
    e = grow_dev(&ws.d_int, &ws.cap_int, ni);
    if (e == cudaSuccess) e = grow_dev(&ws.d_dbl, &ws.cap_dbl, nd);
    if (e != cudaSuccess) return e;
    size_t oi = 0, od = 0;
    for (int k = 0; k < count; ++k) {
        const ReinvJob &j = jobs[k];
        const size_t m = j.m, n = j.n, mn = std::min(m, n) + 1;
        ReinvItem it{};
        it.A = j.A;
        it.b = j.b;
        it.c = j.c;
        it.m = j.m;
        it.n = j.n;
        it.sense = j.sense;
        it.basis = j.basis;
        it.T = j.T;
        it.P = j.P;
        it.x = j.x;
        it.y = j.y;
        it.obj = j.obj;
        int *ib = ws.d_int + oi;
        it.Lflag = ib;
        it.S = ib + m;
        it.R = ib + m + n;
        it.posS = ib + 2 * m + n;
        it.posR = ib + 2 * m + 2 * n;
        it.counts = ws.d_counts + 2 * (size_t)k;
        double *db = ws.d_dbl + od;
        it.xS = db;
        it.yR = db + mn;
        it.zrow = db + 2 * mn;
        it.rhs = db + 2 * mn + n + m;
        it.chk = ws.d_chk + k;
        ws.h_items[k] = it;
        oi += (3 * m + 2 * n + 63) / 64 * 64;
        od += (2 * mn + n + 2 * m + 31) / 32 * 32;
    }
    // the lists of all LPs, and their counts
    e = cudaMemcpyAsync(ws.d_items, ws.h_items, count * sizeof(ReinvItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_reinv_lists_batch(ws.d_items, count, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.h_counts, ws.d_counts, 2 * (size_t)count * sizeof(int),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    // W of the LPs the one-CTA kernel takes
    size_t nw = 0;
    for (int k = 0; k < count; ++k) {
        const int ns = ws.h_counts[2 * k];
        if (ws.h_counts[2 * k + 1] != ns) {
            *bad = k;
            return cudaSuccess;
        }
        if (ns <= kReinvCtaMax) nw += (size_t)ns * (((size_t)2 * ns + 1 + 31) / 32 * 32);
    }
    e = grow_dev(&ws.d_W, &ws.cap_W, std::max<size_t>(nw, 1));
    if (e != cudaSuccess) return e;
    int nb = 0;
    size_t ow = 0;
    std::vector<int> big;
    std::vector<ReinvItem> small;
    for (int k = 0; k < count; ++k) {
        ReinvItem it = ws.h_items[k];
        it.ns = ws.h_counts[2 * k];
        if (it.ns <= kReinvCtaMax) {
            it.Wp = ((long long)2 * it.ns + 1 + 31) / 32 * 32;
            it.W = ws.d_W + ow;
            ow += (size_t)it.ns * it.Wp;
            small.push_back(it);
            ++nb;
        } else {
            big.push_back(k);
        }
    }
    for (int k = 0; k < nb; ++k) ws.h_items[k] = small[k];
    e = cudaMemcpyAsync(ws.d_items, ws.h_items, nb * sizeof(ReinvItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_reinv_solve_batch(prec, ws.d_items, nb, s);
    // the others LP by LP with the multi-CTA kernels and the pool's buffers
    for (int k : big) {
        if (e != cudaSuccess) break;
        const ReinvJob &j = jobs[k];
        const int ns = ws.h_counts[2 * k];
        const size_t needW = (size_t)ns * (((size_t)2 * ns + 1 + 31) / 32 * 32);
        if (needW > rp.cap_W) {
            if (rp.rb.W) cudaFree(rp.rb.W);
            rp.rb.W = nullptr;
            rp.cap_W = 0;
            e = cudaMalloc(&rp.rb.W, needW * sizeof(double));
            if (e != cudaSuccess) break;
            rp.cap_W = needW;
        }
        e = launch_reinv_lists(j.basis, j.m, j.n, rp.rb, s);
        if (e != cudaSuccess) break;
        rp.rb.Wp = ((long long)2 * ns + 1 + 31) / 32 * 32;
        e = launch_reinv_solve(prec, j.A, j.b, j.c, j.sense, j.m, j.n, j.basis, rp.rb, ns, j.T, j.P,
                               j.x, j.y, j.obj, sms, spin_limit, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.d_chk + k, rp.rb.chk, sizeof(ReinvCheck), cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.h_chk, ws.d_chk, count * sizeof(ReinvCheck), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

}  // namespace gbs
