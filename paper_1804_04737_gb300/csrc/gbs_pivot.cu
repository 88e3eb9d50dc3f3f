// Dense tableau simplex kernels for sm_103a.
//
// One persistent grid runs whole pivot sequences (the paper's Step I keeps its
// thread team alive for the whole solve, Sec. 3; here the team is a grid of
// CTAs, one per SM, that never returns to the host between pivots).
//
// Work split.  CTA g owns the column strip [g*W, g*W + W) of every row.  A
// pivot is two phases separated by a grid barrier:
//
//   S (select)  every CTA reduces the selection partials of the previous
//               phase to the entering column q (primal, Sec. 2 Step 2) or the
//               leaving row r (dual simplex); then
//                 primal: ratio test of Step 3 over the CTA's block of rows,
//                         writing per-CTA partials;
//                 dual:   the entering-column ratio over row r, computed
//                         redundantly by every CTA (the row is short);
//               and copies its block of rows of the pivot column into colbuf.
//   U (update)  every CTA reduces the ratio partials to the pivot row p,
//               divides its strip of row p by the pivot (Step 4) into shared
//               memory, and applies T[i][j] = fma(-col[i], prow[j], T[i][j])
//               to its strip of every other row, objective row included
//               (Step 5).  The objective row (primal) or the rhs column
//               (dual) is inspected on the fly, giving the selection partials
//               of the next pivot -- the paper's Step VI fuses the objective
//               row update with the next pricing in the same way.
//
// Race freedom: in phase U a CTA reads and writes only its own strip, plus
// colbuf and the partials, which nobody writes in U.  Row p of the strip is
// read into shared memory before any thread of the CTA writes it.  In phase S
// nothing writes the tableau.  Partials are double-buffered by phase.
//
// Waits are bounded: a barrier that does not complete within the spin limit
// sets the error flag and the kernel returns with status TIMEOUT.

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "gbs_internal.h"

namespace gbs {

namespace {

constexpr int kMaxThreads = 1024;

__device__ __forceinline__ Cand cand_empty() {
    Cand c;
    c.v = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    c.key = 0x7fffffff;
    c.idx = -1;
    return c;
}

__device__ __forceinline__ bool cand_less(const Cand &a, const Cand &b) {
    return a.v < b.v || (a.v == b.v && a.key < b.key);
}

__device__ __forceinline__ void cand_take(Cand &best, double v, int key, int idx) {
    if (v < best.v || (v == best.v && key < best.key)) {
        best.v = v;
        best.key = key;
        best.idx = idx;
    }
}

__device__ __forceinline__ Cand warp_min(Cand c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        Cand d;
        d.v = __shfl_xor_sync(0xffffffffu, c.v, o);
        d.key = __shfl_xor_sync(0xffffffffu, c.key, o);
        d.idx = __shfl_xor_sync(0xffffffffu, c.idx, o);
        if (cand_less(d, c)) c = d;
    }
    return c;
}

// Minimum over the CTA; every thread gets the result.  Uses red[0..32].
__device__ Cand block_min(Cand c, Cand *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    c = warp_min(c);
    __syncthreads();  // red may still be read from a previous call
    if (lane == 0) red[wid] = c;
    __syncthreads();
    if (wid == 0) {
        Cand d = lane < nw ? red[lane] : cand_empty();
        d = warp_min(d);
        if (lane == 0) red[32] = d;
    }
    __syncthreads();
    return red[32];
}

// Minimum of the G partials written by the previous phase (read from L2).
__device__ Cand reduce_partials(const Cand *part, int G, Cand *red) {
    Cand c = cand_empty();
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        Cand d;
        d.v = __ldcg(&part[k].v);
        d.key = __ldcg(&part[k].key);
        d.idx = __ldcg(&part[k].idx);
        if (cand_less(d, c)) c = d;
    }
    return block_min(c, red);
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}

// Grid barrier with a bounded wait.  Returns false (in every thread of the
// CTA) when this or another CTA gave up waiting.
__device__ bool grid_sync(unsigned *bar, int *err, int G, long long spin_limit, int *s_flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (G > 1) {
            unsigned *count = bar;
            unsigned *gen = bar + 32;
            const unsigned g0 = ld_acquire(gen);
            __threadfence();
            const unsigned old = atom_add_acq_rel(count, 1u);
            if (old == (unsigned)G - 1u) {
                atomicExch(count, 0u);
                st_release(gen, g0 + 1u);
            } else {
                const long long t0 = clock64();
                while (ld_acquire(gen) == g0) {
                    if (clock64() - t0 > spin_limit) {
                        atomicExch(err, 1);
                        ok = 0;
                        break;
                    }
                }
            }
            __threadfence();
        }
        if (*(volatile int *)err) ok = 0;
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

template <typename T>
struct Vec;
template <>
struct Vec<double> {
    typedef double2 type;
    static constexpr int W = 2;
};
template <>
struct Vec<float> {
    typedef float4 type;
    static constexpr int W = 4;
};

__device__ __forceinline__ double2 ldv(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ float4 ldv(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ double lds(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float lds(const float *p) { return __ldcg(p); }

__device__ __forceinline__ double getc(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float getc(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// t <- fma(a, pr, t) componentwise (a = -col[i]).
__device__ __forceinline__ void vfma(double2 &t, double a, const double2 &pr) {
    t.x = fma(a, pr.x, t.x);
    t.y = fma(a, pr.y, t.y);
}
__device__ __forceinline__ void vfma(float4 &t, float a, const float4 &pr) {
    t.x = fmaf(a, pr.x, t.x);
    t.y = fmaf(a, pr.y, t.y);
    t.z = fmaf(a, pr.z, t.z);
    t.w = fmaf(a, pr.w, t.w);
}

// Per-thread running candidate of the next selection, fed with freshly
// updated values: the objective row (primal pricing, Sec. 2 Step 2) or the
// rhs column (dual simplex leaving row).
template <typename T, typename V>
__device__ __forceinline__ void watch_row(Cand &best, int sense, int i, int m, int N, int col0,
                                          const V &t, int rhs_lane, double eps_d, double eps_r,
                                          int bland, int p, int q, const int *basis) {
    constexpr int VW = Vec<T>::W;
    if (sense == 0) {
        if (i == m) {
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                const int j = col0 + k;
                const double z = (double)getc(t, k);
                if (j < N - 1 && z < -eps_d) cand_take(best, bland ? 0.0 : z, j, j);
            }
        }
    } else if (rhs_lane >= 0 && i < m) {
        const double v = (double)getc(t, rhs_lane);
        if (v < -eps_r) {
            const int key = bland ? (i == p ? q : __ldcg(basis + i)) : i;
            cand_take(best, bland ? 0.0 : v, key, i);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pivot_kernel(LpDesc *__restrict__ d, int W, long long spin_limit, long long budget) {
    typedef typename Vec<T>::type V;
    constexpr int VW = Vec<T>::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sprow = reinterpret_cast<T *>(smem_raw);
    __shared__ Cand red[33];
    __shared__ int s_flag;

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, B = blockDim.x;

    T *__restrict__ Tab = reinterpret_cast<T *>(d->T);
    T *__restrict__ colbuf = reinterpret_cast<T *>(d->colbuf);
    int *__restrict__ basis = d->basis;
    Cand *part_sel = d->part_sel;
    Cand *part_ratio = d->part_ratio;
    const long long P = d->P;
    const int m = d->m, M = d->M, N = d->N, sense = d->sense;
    const double eps_d = d->eps_d, eps_p = d->eps_p, eps_r = d->eps_r;
    const int bland_after = d->bland_after;
    long long iters = d->iters;
    const long long iter_limit =
        iters > 0x3fffffffffffffffll - budget ? 0x3fffffffffffffffll : iters + budget;
    int deg = d->deg;
    int status = ST_RUNNING;

    // Column strip of this CTA and its row block for the ratio test.
    const int c0 = g * W;  // < P: the host launches ceil(P / W) CTAs
    const int c1 = (int)min((long long)c0 + W, P);
    const int vpr = (c1 - c0) / VW;
    const int rpp = vpr > 0 ? B / vpr : 0;
    const int lr = vpr > 0 ? tid / vpr : 0;
    const int lv = vpr > 0 ? tid - lr * vpr : 0;
    const bool active = vpr > 0 && lr < rpp;
    const int col0 = c0 + lv * VW;
    const int rhs_lane = (active && N - 1 >= col0 && N - 1 < col0 + VW) ? (N - 1 - col0) : -1;
    const int RPC = (M + G - 1) / G;
    const int r0 = min(M, g * RPC), r1 = min(M, r0 + RPC);

    // Selection partials of the current tableau.
    {
        const int bland = deg >= bland_after;
        Cand c = cand_empty();
        if (sense == 0) {
            const T *z = Tab + (long long)m * P;
            for (int j = c0 + tid; j < c1 && j < N - 1; j += B) {
                const double v = (double)lds(z + j);
                if (v < -eps_d) cand_take(c, bland ? 0.0 : v, j, j);
            }
        } else if (N - 1 >= c0 && N - 1 < c1) {
            for (int i = tid; i < m; i += B) {
                const double v = (double)lds(Tab + (long long)i * P + (N - 1));
                if (v < -eps_r) cand_take(c, bland ? 0.0 : v, bland ? __ldcg(basis + i) : i, i);
            }
        }
        c = block_min(c, red);
        if (tid == 0) part_sel[g] = c;
    }
    if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) status = ST_TIMEOUT;

    while (status == ST_RUNNING) {
        // ---------------- phase S: select ----------------
        const int bland = deg >= bland_after;
        const Cand sel = reduce_partials(part_sel, G, red);
        int q = -1, p_dual = -1;
        double rmin_dual = 0.0;
        if (sel.idx < 0) {
            status = ST_OPTIMAL;
            break;
        }
        if (iters >= iter_limit) {
            status = ST_ITER_LIMIT;
            break;
        }
        if (sense == 0) {
            q = sel.idx;
            Cand c = cand_empty();
            for (int i = r0 + tid; i < r1; i += B) {
                const T a = lds(Tab + (long long)i * P + q);
                colbuf[i] = a;
                if (i < m && (double)a > eps_p) {
                    const T rhs = lds(Tab + (long long)i * P + (N - 1));
                    const T r = (rhs > (T)0 ? rhs : (T)0) / a;
                    cand_take(c, (double)r, bland ? __ldcg(basis + i) : i, i);
                }
            }
            c = block_min(c, red);
            if (tid == 0) part_ratio[g] = c;
        } else {
            p_dual = sel.idx;
            const T *rowr = Tab + (long long)p_dual * P;
            const T *z = Tab + (long long)m * P;
            Cand c = cand_empty();
            for (int j = tid; j < N - 1; j += B) {
                const T a = lds(rowr + j);
                if ((double)a < -eps_p) {
                    const T zj = lds(z + j);
                    const T t = (zj > (T)0 ? zj : (T)0) / (-a);
                    cand_take(c, (double)t, j, j);
                }
            }
            c = block_min(c, red);
            if (c.idx < 0) {
                status = ST_INFEASIBLE;
                break;
            }
            q = c.idx;
            rmin_dual = c.v;
            for (int i = r0 + tid; i < r1; i += B) colbuf[i] = lds(Tab + (long long)i * P + q);
        }
        if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) {
            status = ST_TIMEOUT;
            break;
        }

        // ---------------- phase U: update ----------------
        int p;
        double rmin;
        if (sense == 0) {
            const Cand rc = reduce_partials(part_ratio, G, red);
            if (rc.idx < 0) {
                status = ST_UNBOUNDED;
                break;
            }
            p = rc.idx;
            rmin = rc.v;
        } else {
            p = p_dual;
            rmin = rmin_dual;
        }
        deg = (rmin == 0.0) ? deg + 1 : 0;
        if (g == 0 && tid == 0) {
            if (iters < d->trace_cap) {
                d->trace[2 * iters] = p;
                d->trace[2 * iters + 1] = q;
            }
            basis[p] = q;
            d->last_p = p;
            d->last_q = q;
        }
        const T piv = lds(colbuf + p);
        const T *rowp = Tab + (long long)p * P;
        for (int j = c0 + tid; j < c1; j += B) sprow[j - c0] = lds(rowp + j) / piv;
        __syncthreads();

        const int nbland = deg >= bland_after;  // rule of the next selection
        Cand watch = cand_empty();
        if (active) {
            const V pr = *reinterpret_cast<const V *>(sprow + lv * VW);
            T *base = Tab + col0;
            int i = lr;
            for (; i + 3 * rpp < M; i += 4 * rpp) {
                const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                V *p0 = reinterpret_cast<V *>(base + (long long)i * P);
                V *p1 = reinterpret_cast<V *>(base + (long long)i1 * P);
                V *p2 = reinterpret_cast<V *>(base + (long long)i2 * P);
                V *p3 = reinterpret_cast<V *>(base + (long long)i3 * P);
                V t0 = ldv(p0), t1 = ldv(p1), t2 = ldv(p2), t3 = ldv(p3);
                const T a0 = -lds(colbuf + i), a1 = -lds(colbuf + i1);
                const T a2 = -lds(colbuf + i2), a3 = -lds(colbuf + i3);
                if (i == p) t0 = pr; else vfma(t0, a0, pr);
                if (i1 == p) t1 = pr; else vfma(t1, a1, pr);
                if (i2 == p) t2 = pr; else vfma(t2, a2, pr);
                if (i3 == p) t3 = pr; else vfma(t3, a3, pr);
                *p0 = t0;
                *p1 = t1;
                *p2 = t2;
                *p3 = t3;
                watch_row<T>(watch, sense, i, m, N, col0, t0, rhs_lane, eps_d, eps_r, nbland, p, q, basis);
                watch_row<T>(watch, sense, i1, m, N, col0, t1, rhs_lane, eps_d, eps_r, nbland, p, q, basis);
                watch_row<T>(watch, sense, i2, m, N, col0, t2, rhs_lane, eps_d, eps_r, nbland, p, q, basis);
                watch_row<T>(watch, sense, i3, m, N, col0, t3, rhs_lane, eps_d, eps_r, nbland, p, q, basis);
            }
            for (; i < M; i += rpp) {
                V *p0 = reinterpret_cast<V *>(base + (long long)i * P);
                V t0 = ldv(p0);
                const T a0 = -lds(colbuf + i);
                if (i == p) t0 = pr; else vfma(t0, a0, pr);
                *p0 = t0;
                watch_row<T>(watch, sense, i, m, N, col0, t0, rhs_lane, eps_d, eps_r, nbland, p, q, basis);
            }
        }
        watch = block_min(watch, red);
        if (tid == 0) part_sel[g] = watch;
        ++iters;
        if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) {
            status = ST_TIMEOUT;
            break;
        }
    }

    if (g == 0 && tid == 0) {
        d->status = (*(volatile int *)d->err) ? ST_TIMEOUT : status;
        d->iters = iters;
        d->iter_limit = iter_limit;
        d->deg = deg;
    }
}

// ---------------------------------------------------------------------------

__device__ __forceinline__ void atomic_max_bits(unsigned long long *p, double v) {
    atomicMax(p, (unsigned long long)__double_as_longlong(fabs(v)));
}

// max |A|, max |b|, max |c| (as bit patterns of non-negative doubles, whose
// unsigned order is the numeric order), sign and finiteness flags.
__global__ void inspect_kernel(const double *__restrict__ A, const double *__restrict__ b,
                               const double *__restrict__ c, int m, int n, InputStats *out) {
    const long long total = (long long)m * n;
    double amax = 0.0, bmax = 0.0, cmax = 0.0;
    int flags = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += stride) {
        const double v = A[k];
        if (!isfinite(v)) flags |= 4;
        amax = fmax(amax, fabs(v));
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += stride) {
        const double v = b[k];
        if (!isfinite(v)) flags |= 4;
        if (v < 0.0) flags |= 1;
        bmax = fmax(bmax, fabs(v));
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride) {
        const double v = c[k];
        if (!isfinite(v)) flags |= 4;
        if (v < 0.0) flags |= 2;
        cmax = fmax(cmax, fabs(v));
    }
    if (flags & 4) {  // keep the maxima meaningful even with NaN around
        amax = isfinite(amax) ? amax : 0.0;
        bmax = isfinite(bmax) ? bmax : 0.0;
        cmax = isfinite(cmax) ? cmax : 0.0;
    }
    if (amax > 0.0) atomic_max_bits(&out->amax_bits, amax);
    if (bmax > 0.0) atomic_max_bits(&out->bmax_bits, bmax);
    if (cmax > 0.0) atomic_max_bits(&out->cmax_bits, cmax);
    if (flags) atomicOr(&out->flags, flags);
}

// Sec. 2 Step 1: the initial tableau (rows [A | I | b], objective row
// [-c | 0 | 0]; dual form [-A | I | -b] and [c | 0 | 0]), padded with zeros
// to the pitch P.
template <typename T>
__global__ void build_kernel(const double *__restrict__ A, const double *__restrict__ b,
                             const double *__restrict__ c, int m, int n, int sense,
                             T *__restrict__ Tab, long long P, int *__restrict__ basis) {
    const int N = n + m + 1;
    const long long total = (long long)(m + 1) * P;
    const double sg = sense == 0 ? 1.0 : -1.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += stride) {
        const int i = (int)(k / P);
        const int j = (int)(k - (long long)i * P);
        double v = 0.0;
        if (i < m) {
            if (j < n) v = sg * A[(long long)i * n + j];
            else if (j == n + i) v = 1.0;
            else if (j == N - 1) v = sg * b[i];
        } else if (j < n) {
            v = -sg * c[j];
        }
        Tab[k] = (T)v;
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += stride)
        basis[k] = n + (int)k;
}

// Solution read-off, part 1: zero x, duals from the objective row, objective.
template <typename T>
__global__ void extract_kernel1(const T *__restrict__ Tab, int m, int n, long long P, int sense,
                                double *x, double *y, double *obj) {
    const int N = n + m + 1;
    const T *z = Tab + (long long)m * P;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += stride)
        x[k] = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += stride)
        y[k] = (double)z[n + k];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const double zv = (double)z[N - 1];
        *obj = sense == 0 ? zv : -zv;
    }
}

// Part 2: x_j = rhs of the row where j is basic.
template <typename T>
__global__ void extract_kernel2(const T *__restrict__ Tab, const int *__restrict__ basis, int m,
                                int n, long long P, double *x) {
    const int N = n + m + 1;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += stride) {
        const int j = basis[i];
        if (j < n) x[j] = (double)Tab[i * P + (N - 1)];
    }
}

__global__ void to_fp64_kernel(const float *__restrict__ Tab, long long P, int M, int N,
                               double *__restrict__ out) {
    const long long total = (long long)M * N;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += stride) {
        const long long i = k / N, j = k - i * N;
        out[k] = (double)Tab[i * P + j];
    }
}

int grid_for(long long work, int threads) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_inspect(const double *A, const double *b, const double *c, int m, int n,
                           InputStats *out, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(InputStats), s);
    if (e != cudaSuccess) return e;
    const long long work = (long long)m * n;
    inspect_kernel<<<grid_for(work, 256), 256, 0, s>>>(A, b, c, m, n, out);
    return cudaGetLastError();
}

cudaError_t launch_build(int prec, const double *A, const double *b, const double *c, int m,
                         int n, int sense, void *T, long long P, int *basis, cudaStream_t s) {
    const long long work = (long long)(m + 1) * P;
    if (prec == PREC_FP64)
        build_kernel<double><<<grid_for(work, 256), 256, 0, s>>>(A, b, c, m, n, sense,
                                                                 (double *)T, P, basis);
    else
        build_kernel<float><<<grid_for(work, 256), 256, 0, s>>>(A, b, c, m, n, sense,
                                                                (float *)T, P, basis);
    return cudaGetLastError();
}

PivotShape choose_shape(int prec, int M, long long P, int sms, int threads, int ctas) {
    PivotShape sh;
    const int vw = prec == PREC_FP64 ? 2 : 4;       // elements per 16-byte vector
    const int sector = prec == PREC_FP64 ? 4 : 8;   // elements per 32-byte sector
    sh.threads = threads > 0 ? threads : kMaxThreads;
    if (sh.threads > kMaxThreads) sh.threads = kMaxThreads;
    if (sh.threads < 64) sh.threads = 64;
    sh.threads = (sh.threads + 31) / 32 * 32;
    long long g;
    if (ctas > 0) {
        g = ctas;
    } else {
        // enough CTAs to keep ~32K elements each, at most one per SM
        g = ((long long)M * P + 32767) / 32768;
        if (g > sms) g = sms;
    }
    // a strip must fit one pass of the CTA: columns <= threads * vw
    const long long gmin = (P + (long long)sh.threads * vw - 1) / ((long long)sh.threads * vw);
    if (g < gmin) g = gmin;
    if (g < 1) g = 1;
    long long w = (P + g - 1) / g;
    w = (w + sector - 1) / sector * sector;
    sh.strip = (int)w;
    sh.ctas = (int)((P + w - 1) / w);
    return sh;
}

cudaError_t launch_pivot(int prec, LpDesc *d_desc, const PivotShape &sh, long long spin_limit,
                         long long budget, cudaStream_t s) {
    const size_t esz = prec == PREC_FP64 ? sizeof(double) : sizeof(float);
    size_t smem = (size_t)sh.strip * esz;
    int W = sh.strip;
    void *args[] = {&d_desc, &W, &spin_limit, &budget};
    const void *fn = prec == PREC_FP64 ? (const void *)pivot_kernel<double>
                                       : (const void *)pivot_kernel<float>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    // A cooperative launch fails instead of running when the grid cannot be
    // co-resident, which the grid barrier needs.
    return cudaLaunchCooperativeKernel(fn, dim3(sh.ctas), dim3(sh.threads), args, smem, s);
}

cudaError_t launch_extract(int prec, const LpDesc *, const void *T, const int *basis, int m,
                           int n, long long P, int sense, double *x, double *y, double *obj,
                           cudaStream_t s) {
    const long long work = (long long)(m > n ? m : n);
    if (prec == PREC_FP64) {
        extract_kernel1<double><<<grid_for(work, 256), 256, 0, s>>>((const double *)T, m, n, P,
                                                                    sense, x, y, obj);
        extract_kernel2<double><<<grid_for(m, 256), 256, 0, s>>>((const double *)T, basis, m, n,
                                                                 P, x);
    } else {
        extract_kernel1<float><<<grid_for(work, 256), 256, 0, s>>>((const float *)T, m, n, P,
                                                                   sense, x, y, obj);
        extract_kernel2<float><<<grid_for(m, 256), 256, 0, s>>>((const float *)T, basis, m, n,
                                                                P, x);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_fp64(const float *T, long long P, int M, int N, double *out,
                           cudaStream_t s) {
    to_fp64_kernel<<<grid_for((long long)M * N, 256), 256, 0, s>>>(T, P, M, N, out);
    return cudaGetLastError();
}

}  // namespace gbs
