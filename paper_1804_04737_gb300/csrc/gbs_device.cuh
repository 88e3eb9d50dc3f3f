// Device helpers shared by the pivot and reinversion kernels: ordered keys,
// candidate reductions, bounded grid barrier and counter waits, vector types.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbs_internal.h"

namespace gbs {
namespace dev {

// ---------------------------------------------------------------------------
// Ordered keys.  GB300 runs FP64 compares and min/max on its narrow FP64 pipe
// (the same two operations per SM per clock as an FP64 FMA), so selection
// compares doubles through order-preserving integer keys instead: for any two
// non-NaN values, x < y exactly when okey(x) < okey(y).

constexpr unsigned long long kSign = 0x8000000000000000ull;

__device__ __forceinline__ unsigned long long okey(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    return (u & kSign) ? ~u : (u | kSign);
}
__device__ __forceinline__ unsigned long long okey(float x) {
    const unsigned u = __float_as_uint(x);
    return (u & 0x80000000u) ? (unsigned long long)(~u) : (unsigned long long)(u | 0x80000000u);
}

__device__ __forceinline__ Cand cand_empty() {
    Cand c;
    c.vk = ~0ull;
    c.key = 0x7fffffff;
    c.idx = -1;
    return c;
}

__device__ __forceinline__ bool cand_less(const Cand &a, const Cand &b) {
    return a.vk < b.vk || (a.vk == b.vk && a.key < b.key);
}

__device__ __forceinline__ void cand_take(Cand &best, unsigned long long vk, int key, int idx) {
    if (vk < best.vk || (vk == best.vk && key < best.key)) {
        best.vk = vk;
        best.key = key;
        best.idx = idx;
    }
}

// Warp-wide minima on the redux unit: one instruction per 32-bit minimum.  A
// five-step shuffle butterfly took several microseconds on GB300 while the
// SM's load/store path was busy with the tableau stream.
__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
    const unsigned hi = (unsigned)(v >> 32);
    const unsigned mhi = __reduce_min_sync(0xffffffffu, hi);
    const unsigned mlo = __reduce_min_sync(0xffffffffu, hi == mhi ? (unsigned)v : 0xffffffffu);
    return ((unsigned long long)mhi << 32) | mlo;
}

// Lowest lane holding the lexicographic minimum of (vk, key), keys >= 0;
// the minimum itself in *mvk, *mkey.
__device__ __forceinline__ int warp_argmin(unsigned long long vk, int key, unsigned long long *mvk,
                                           int *mkey) {
    const unsigned long long m = warp_min_u64(vk);
    const bool at = vk == m;
    const unsigned k = __reduce_min_sync(0xffffffffu, at ? (unsigned)key : 0xffffffffu);
    const unsigned bal = __ballot_sync(0xffffffffu, at && (unsigned)key == k);
    *mvk = m;
    *mkey = (int)k;
    return __ffs(bal) - 1;
}

// Warp-wide candidate minimum; every lane gets it.
__device__ __forceinline__ Cand warp_min(Cand c) {
    Cand r;
    const int src = warp_argmin(c.vk, c.key, &r.vk, &r.key);
    r.idx = __shfl_sync(0xffffffffu, c.idx, src);
    return r;
}

// Block-wide candidate minimum; every thread gets the result.  `buf` (32
// entries) belongs to one call site; one __syncthreads.
__device__ __forceinline__ Cand block_min_c(Cand c, Cand *buf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    c = warp_min(c);
    if (lane == 0) buf[wid] = c;
    __syncthreads();
    Cand r = buf[0];
    for (int k = 1; k < nw; ++k)
        if (cand_less(buf[k], r)) r = buf[k];
    return r;
}

__device__ __forceinline__ unsigned long long block_min_u(unsigned long long v,
                                                          unsigned long long *buf) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    v = warp_min_u64(v);
    if (lane == 0) buf[wid] = v;
    __syncthreads();
    unsigned long long r = buf[0];
    for (int k = 1; k < nw; ++k) r = buf[k] < r ? buf[k] : r;
    return r;
}

__device__ __forceinline__ Cand load_partials_min(const Cand *part, int G, Cand *buf) {
    Cand c = cand_empty();
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        Cand e;
        e.vk = __ldcg(&part[k].vk);
        e.key = __ldcg(&part[k].key);
        e.idx = __ldcg(&part[k].idx);
        if (cand_less(e, c)) c = e;
    }
    return block_min_c(c, buf);
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

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid barrier with a bounded wait.  Returns false (in every thread of the
// CTA) when this or another CTA gave up waiting.
static __device__ bool grid_sync(unsigned *bar, int *err, int G, long long spin_limit, int *s_flag) {
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
                    if (clock64() - t0 > spin_limit || *(volatile int *)err) {
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

// Wait (thread 0, bounded) until *ctr has reached target.  False when the
// wait ran out or another CTA reported a timeout.
static __device__ bool wait_count(unsigned *ctr, unsigned target, int *err, long long spin_limit,
                           int *s_flag) {
    if (threadIdx.x == 0) {
        int ok = 1;
        const long long t0 = clock64();
        while ((int)(ld_acquire(ctr) - target) < 0) {
            if (clock64() - t0 > spin_limit || *(volatile int *)err) {
                atomicExch(err, 1);
                ok = 0;
                break;
            }
        }
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

// The host's abort word (mapped host memory; nullptr: none).  The load is
// issued where this is called and its value used later, so its latency (a
// round trip to host memory) overlaps the work in between.
__device__ __forceinline__ int abort_peek(const int *a) {
    int v = 0;
    if (a) asm volatile("ld.relaxed.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__device__ __forceinline__ double2 ldv(const double2 *p) { return __ldcg(p); }
__device__ __forceinline__ float4 ldv(const float4 *p) { return __ldcg(p); }
__device__ __forceinline__ double lds(const double *p) { return __ldcg(p); }
__device__ __forceinline__ float lds(const float *p) { return __ldcg(p); }

__device__ __forceinline__ double getc(const double2 &v, int k) { return k == 0 ? v.x : v.y; }
__device__ __forceinline__ float getc(const float4 &v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

// t <- fma(-c, pr, t) componentwise (Sec. 2 Step 5 on one vector).
__device__ __forceinline__ void vfma(double2 &t, double c, const double2 &pr) {
    t.x = fma(-c, pr.x, t.x);
    t.y = fma(-c, pr.y, t.y);
}
__device__ __forceinline__ void vfma(float4 &t, float c, const float4 &pr) {
    t.x = fmaf(-c, pr.x, t.x);
    t.y = fmaf(-c, pr.y, t.y);
    t.z = fmaf(-c, pr.z, t.z);
    t.w = fmaf(-c, pr.w, t.w);
}

// (x > 0 ? x : 0) and -x through the sign bit, off the FP64 pipe.
__device__ __forceinline__ double pos_part(double x) {
    return __double_as_longlong(x) > 0 ? x : 0.0;
}
__device__ __forceinline__ float pos_part(float x) { return __float_as_int(x) > 0 ? x : 0.0f; }
__device__ __forceinline__ double neg(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)kSign);
}
__device__ __forceinline__ float neg(float x) { return __int_as_float(__float_as_int(x) ^ 0x80000000); }

// Screening key of num / den (num >= +0, den > 0): okey of a value within a
// relative 2^-20 of the exact quotient.  In range it is one single-precision
// division of the truncated operands (integer ops convert in both
// directions); outside it, the exact division.  Every row whose exactly
// rounded quotient could be the minimum has a screening value within
// kScreen of the smallest screening value, so screening never drops the row
// the exact ratios select (ties included).
__device__ __forceinline__ float trunc_to_float(long long b) {  // positive, exponent in range
    const int e = (int)(b >> 52) - 1023 + 127;
    return __int_as_float((e << 23) | (int)((b >> 29) & 0x7fffff));
}
__device__ __forceinline__ unsigned long long screen_key(double num, double den) {
    const long long nb = __double_as_longlong(num), db = __double_as_longlong(den);
    if (nb == 0) return okey(0.0);
    const int ne = (int)(nb >> 52), de = (int)(db >> 52);
    if (ne >= 1023 - 60 && ne <= 1023 + 60 && de >= 1023 - 60 && de <= 1023 + 60) {
        const float q = __fdividef(trunc_to_float(nb), trunc_to_float(db));
        const unsigned qb = __float_as_uint(q);  // positive normal: quotient in [2^-121, 2^121]
        const unsigned long long r =
            ((unsigned long long)(((qb >> 23) & 0xffu) - 127u + 1023u) << 52) |
            ((unsigned long long)(qb & 0x7fffffu) << 29);
        return r | kSign;
    }
    return okey(num / den);
}
__device__ __forceinline__ unsigned long long screen_key(float num, float den) {
    const int nb = __float_as_int(num), db = __float_as_int(den);
    if (nb == 0) return okey(0.0f);
    const int ne = nb >> 23, de = db >> 23;
    if (ne >= 127 - 60 && ne <= 127 + 60 && de >= 127 - 60 && de <= 127 + 60)
        return okey(__fdividef(num, den));
    return okey(num / den);
}
// Screening threshold: okey(rstar * kScreen) for a screening key rstar.
constexpr double kScreen = 1.0 + 1.0 / 65536.0;  // 1 + 2^-16
__device__ __forceinline__ unsigned long long screen_thr(unsigned long long rk, double) {
    const double r = __longlong_as_double((long long)(rk & ~kSign));
    return okey(r * kScreen);
}
__device__ __forceinline__ unsigned long long screen_thr(unsigned long long rk, float) {
    const float r = __uint_as_float((unsigned)(rk & 0x7fffffffu));
    return okey(r * (float)kScreen);
}

// One 16-byte vector of row i: Step 4 for the pivot row, Step 5 otherwise.
template <typename T, typename V>
__device__ __forceinline__ V pivot_vec(const V &t, int i, int p, T col_i, const V &pr) {
    if (i == p) return pr;
    V r = t;
    vfma(r, col_i, pr);
    return r;
}

}  // namespace dev
}  // namespace gbs
