// Batched solves (lp_solve_batch): many independent LPs pivoted in one
// persistent launch.
//
// Layout in HBM: the inputs of all LPs packed in one FP64 array; every LP's
// pitched tableau in one arena; per-LP descriptors, bases, partials and
// barrier words in small arrays.  The launch's CTAs pop (lp, rank) work items
// in order, largest LPs first, and each LP is solved by a group of CTAs sized
// to its tableau (group_elems tableau elements per CTA), so a 1024 x 1024 LP
// and a 32 x 32 LP finish in comparable times.  Device memory is kept in a
// per-device grow-only pool between calls.
//
// Per-LP arithmetic is exactly the single-LP kernel's (same device function),
// so every LP's pivots and results are bit for bit those of solving it alone.

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gbs_device.cuh"
#include "gbs_internal.h"
#include "gbsimplex.h"

namespace gbs {
namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------- kernels --

struct BatchArrays {
    const long long *in_off;   // per LP: offset of A (then b, then c) in the packed inputs
    const long long *t_off;    // per LP: byte offset of the tableau in the arena
    const long long *xy_off;   // per LP: offset of x (then y) in the packed outputs
    const int *m, *n;
    const int *sense;
    const long long *P;
};

// Packed inputs from caller device pointers: block y = one array (A, b or c
// of LP y/3).
__global__ void batch_gather_kernel(const double *const *src, const long long *dst_off,
                                    const long long *len, double *dst) {
    const int a = blockIdx.y;
    const double *s = src[a];
    double *d = dst + dst_off[a];
    const long long L = len[a];
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < L;
         k += (long long)gridDim.x * blockDim.x)
        d[k] = s[k];
}

__device__ __forceinline__ void atomic_max_abs(unsigned long long *p, double v) {
    if (v > 0.0) atomicMax(p, (unsigned long long)__double_as_longlong(v));
}

// Input statistics per LP (block y = LP): max |A|, |b|, |c|, sign and
// finiteness flags, like the single-LP inspection.
__global__ void batch_inspect_kernel(BatchArrays ba, const double *in, InputStats *stats) {
    const int k = blockIdx.y;
    const int m = ba.m[k], n = ba.n[k];
    const double *A = in + ba.in_off[k], *b = A + (long long)m * n, *c = b + m;
    double amax = 0.0, bmax = 0.0, cmax = 0.0;
    int flags = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long e = t0; e < (long long)m * n; e += stride) {
        const double v = A[e];
        if (!isfinite(v)) flags |= 4; else amax = fmax(amax, fabs(v));
    }
    for (long long e = t0; e < m; e += stride) {
        const double v = b[e];
        if (!isfinite(v)) flags |= 4; else bmax = fmax(bmax, fabs(v));
        if (v < 0.0) flags |= 1;
    }
    for (long long e = t0; e < n; e += stride) {
        const double v = c[e];
        if (!isfinite(v)) flags |= 4; else cmax = fmax(cmax, fabs(v));
        if (v < 0.0) flags |= 2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        cmax = fmax(cmax, __shfl_xor_sync(0xffffffffu, cmax, o));
        flags |= __shfl_xor_sync(0xffffffffu, flags, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_abs(&stats[k].amax_bits, amax);
        atomic_max_abs(&stats[k].bmax_bits, bmax);
        atomic_max_abs(&stats[k].cmax_bits, cmax);
        if (flags) atomicOr(&stats[k].flags, flags);
    }
}

// Sec. 2 Step 1 for every LP (block y = LP), the same values as the
// single-LP build.
template <typename T>
__global__ void batch_build_kernel(BatchArrays ba, const double *in, unsigned char *arena,
                                   int *const *basis_ptr) {
    const int k = blockIdx.y;
    const int m = ba.m[k], n = ba.n[k], N = n + m + 1;
    const long long P = ba.P[k];
    const double *A = in + ba.in_off[k], *b = A + (long long)m * n, *c = b + m;
    T *Tab = reinterpret_cast<T *>(arena + ba.t_off[k]);
    const double sg = ba.sense[k] == 0 ? 1.0 : -1.0;
    const long long total = (long long)(m + 1) * P;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += stride) {
        const int i = (int)(e / P);
        const int j = (int)(e - (long long)i * P);
        double v = 0.0;
        if (i < m) {
            if (j < n) v = sg * A[(long long)i * n + j];
            else if (j == n + i) v = 1.0;
            else if (j == N - 1) v = sg * b[i];
        } else if (j < n) {
            v = -sg * c[j];
        }
        Tab[e] = (T)v;
    }
    int *basis = basis_ptr[k];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < m; e += stride)
        basis[e] = n + (int)e;
}

// Solution read-off for every LP (one block per LP): x, y and the objective.
template <typename T>
__global__ void batch_extract_kernel(BatchArrays ba, const unsigned char *arena,
                                     int *const *basis_ptr, double *xy, double *obj) {
    const int k = blockIdx.x;
    const int m = ba.m[k], n = ba.n[k], N = n + m + 1;
    const long long P = ba.P[k];
    const T *Tab = reinterpret_cast<const T *>(arena + ba.t_off[k]);
    const T *z = Tab + (long long)m * P;
    double *x = xy + ba.xy_off[k], *y = x + n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) x[j] = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) y[i] = (double)z[n + i];
    __syncthreads();
    const int *basis = basis_ptr[k];
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
        const int j = basis[i];
        if (j < n) x[j] = (double)Tab[(long long)i * P + (N - 1)];
    }
    if (threadIdx.x == 0) {
        const double zv = (double)z[N - 1];
        obj[k] = ba.sense[k] == 0 ? zv : -zv;
    }
}

// ------------------------------------------------------------ device pool --

struct Pool {
    std::mutex mu;
    void *dev = nullptr;
    size_t dev_cap = 0;
    void *pin = nullptr;
    size_t pin_cap = 0;
};
Pool g_pool[64];

cudaError_t pool_dev(Pool &p, size_t bytes, void **out) {
    if (bytes > p.dev_cap) {
        if (p.dev) cudaFree(p.dev);
        p.dev = nullptr;
        p.dev_cap = 0;
        cudaError_t e = cudaMalloc(&p.dev, bytes);
        if (e != cudaSuccess) return e;
        p.dev_cap = bytes;
    }
    *out = p.dev;
    return cudaSuccess;
}

cudaError_t pool_pin(Pool &p, size_t bytes, void **out) {
    if (bytes > p.pin_cap) {
        if (p.pin) cudaFreeHost(p.pin);
        p.pin = nullptr;
        p.pin_cap = 0;
        cudaError_t e = cudaMallocHost(&p.pin, bytes);
        if (e != cudaSuccess) return e;
        p.pin_cap = bytes;
    }
    *out = p.pin;
    return cudaSuccess;
}

}  // namespace
}  // namespace gbs

namespace gbs {
namespace {

struct BatchStats {
    double kernel_ms = 0.0;
    long long pivots = 0;
    int ctas = 0, threads = 0, items = 0, max_group = 0;
};
std::mutex g_stats_mu;
BatchStats g_last;

lp_err bfail(lp_err code, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error_global(msg);
    return code;
}

#define B_TRY(call)                                                                    \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return bfail(e_ == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,   \
                         "%s failed: %s", #call, cudaGetErrorString(e_));              \
    } while (0)

}  // namespace
}  // namespace gbs

using namespace gbs;

namespace {

// ------------------------------------------------- FP32 batches (A9 + A11) --

// What the FP32 rounds need of lp_solve_batch's layout.
struct BatchFp32 {
    int count;
    const int *m, *n, *sv, *G, *order;
    const long long *in_off, *t_off, *xy_off, *P;
    const double *d_in;
    unsigned char *d_T;
    double *d_xy, *d_obj;
    LpDesc *h_desc, *d_desc;
    int2 *h_items, *d_items;
    unsigned *d_queue;
    unsigned char *d_bar;
    int ctas, threads, use_smem, sms;
    size_t smem;
    const lp_options *opt;
    cudaStream_t s;
};

// FP32 batch: rounds of one batched launch (every unfinished LP pivots up to
// reinv_k times in FP32), then, LP by LP, the FP64 reinversion of its basis
// and the same decisions as the single-LP FP32 mode: accept an FP32 optimum
// only when the FP64 values are primal and dual feasible, otherwise continue
// with the rule whose invariant holds (primal simplex from a primal-feasible
// basis, dual simplex from a dual-feasible one).  x, y and the objective are
// the FP64 values of the last reinversion.
lp_err solve_batch_fp32(const BatchFp32 &f, lp_status *fin, double *kernel_ms) {
    const int count = f.count;
    cudaStream_t s = f.s;
    size_t cap = 0, capW = 0;
    for (int k = 0; k < count; ++k) {
        cap = std::max(cap, (size_t)std::max(f.m[k], f.n[k]) + f.m[k]);
        const size_t ns = (size_t)std::min(f.m[k], f.n[k]);
        capW = std::max(capW, ns * (((2 * ns + 1) + 31) / 32 * 32));
    }
    ReinvPool rp;
    B_TRY(rp.init(cap));
    B_TRY(cudaMalloc(&rp.rb.W, std::max<size_t>(capW, 1) * sizeof(double)));
    rp.cap_W = capW;
    BatchReinv ws;

    std::vector<int> active(count, 1), rule(count), failed(count, 0);
    std::vector<long long> remaining(count), guard(count), before(count);
    for (int k = 0; k < count; ++k) {
        rule[k] = f.sv[k];
        remaining[k] = f.opt->max_iters;
        guard[k] = 20ll * (f.m[k] + f.n[k]) + 1000;
    }
    cudaEvent_t e0, e1;
    B_TRY(cudaEventCreate(&e0));
    B_TRY(cudaEventCreate(&e1));
    *kernel_ms = 0.0;
    for (int round = 0;; ++round) {
        // work items of the unfinished LPs, largest first
        int nitems = 0;
        long long budget = f.opt->reinv_k;
        for (int o = 0; o < count; ++o) {
            const int k = f.order[o];
            if (!active[k]) continue;
            budget = std::min(budget, remaining[k]);
            for (int r = 0; r < f.G[k]; ++r) f.h_items[nitems++] = make_int2(k, r);
            f.h_desc[k].sense = rule[k];
            before[k] = f.h_desc[k].iters;
        }
        if (nitems == 0) break;
        B_TRY(cudaMemcpyAsync(f.d_items, f.h_items, nitems * sizeof(int2), cudaMemcpyHostToDevice, s));
        B_TRY(cudaMemcpyAsync(f.d_desc, f.h_desc, count * sizeof(LpDesc), cudaMemcpyHostToDevice, s));
        B_TRY(cudaMemsetAsync(f.d_bar, 0, (size_t)count * 512, s));
        B_TRY(cudaMemsetAsync(f.d_queue, 0, sizeof(unsigned), s));
        B_TRY(cudaEventRecord(e0, s));
        B_TRY(launch_batch(PREC_FP32, f.d_desc, f.d_items, nitems, f.d_queue, f.ctas, f.threads,
                           f.smem, f.use_smem, f.opt->spin_timeout_cycles, budget, s));
        B_TRY(cudaEventRecord(e1, s));
        B_TRY(cudaMemcpyAsync(f.h_desc, f.d_desc, count * sizeof(LpDesc), cudaMemcpyDeviceToHost, s));
        B_TRY(cudaStreamSynchronize(s));
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        *kernel_ms += t;
        // the FP64 reinversion of every unfinished LP's basis, batched
        std::vector<int> idx;
        std::vector<ReinvJob> jobs;
        for (int k = 0; k < count; ++k) {
            if (!active[k]) continue;
            LpDesc &d = f.h_desc[k];
            const long long made = d.iters - before[k];
            remaining[k] -= made;
            guard[k] -= made;
            if (d.status == LP_TIMEOUT) {
                fin[k] = LP_TIMEOUT;
                active[k] = 0;
                continue;
            }
            const int m = f.m[k], n = f.n[k];
            const double *A = f.d_in + f.in_off[k], *b = A + (long long)m * n, *c = b + m;
            double *x = f.d_xy + f.xy_off[k];
            jobs.push_back(ReinvJob{A, b, c, m, n, f.sv[k], d.basis, f.d_T + f.t_off[k], f.P[k], x,
                                    x + n, f.d_obj + k});
            idx.push_back(k);
        }
        int badj = -1;
        B_TRY(reinvert_many(PREC_FP32, jobs.data(), (int)jobs.size(), ws, rp, f.sms,
                            f.opt->spin_timeout_cycles, s, &badj));
        if (badj >= 0)
            return bfail(LP_ERR_STATE, "lp_solve_batch: LP %d: inconsistent basis", idx[badj]);
        for (size_t q = 0; q < idx.size(); ++q) {
            const int k = idx[q];
            LpDesc &d = f.h_desc[k];
            const int st = d.status;
            const ReinvCheck *chk = ws.h_chk + q;
            auto finish = [&](lp_status v) {
                fin[k] = v;
                active[k] = 0;
            };
            if (chk->singular) {
                finish(LP_NUMERICAL);
                continue;
            }
            const bool pfeas = key_to_double(chk->rhsmin_key) >= -d.eps_r;
            const bool dfeas = key_to_double(chk->zmin_key) >= -d.eps_d;
            if (st == LP_OPTIMAL) {
                if (pfeas && dfeas) {
                    finish(LP_OPTIMAL);
                } else if ((!pfeas && !dfeas) || ++failed[k] > 4) {
                    finish(LP_NUMERICAL);
                } else {
                    rule[k] = pfeas ? 0 : 1;
                }
                continue;
            }
            if (st == LP_UNBOUNDED || st == LP_INFEASIBLE) {
                finish((lp_status)st);
                continue;
            }
            if (remaining[k] <= 0) {
                finish(LP_ITER_LIMIT);
                continue;
            }
            if (guard[k] <= 0) {
                finish(LP_NUMERICAL);
                continue;
            }
            if (rule[k] == 0 && !pfeas && dfeas) rule[k] = 1;
            else if (rule[k] == 1 && !dfeas && pfeas) rule[k] = 0;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return LP_OK;
}

}  // namespace

extern "C" lp_err lp_solve_batch(int count, const int *m, const int *n, const double *const *A,
                                 const double *const *b, const double *const *c,
                                 const int *sense, const lp_options *opt, double *obj,
                                 lp_status *status, long long *iters, double *const *x,
                                 double *const *y) {
    if (count < 1 || !m || !n || !A || !b || !c)
        return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: need count >= 1 and non-NULL arrays");
    lp_options o;
    if (opt) o = *opt; else lp_options_default(&o);
    if (o.precision != LP_FP64 && o.precision != LP_FP32_REINV)
        return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: unknown precision %d", o.precision);
    if (o.precision == LP_FP32_REINV && o.reinv_k < 1)
        return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: reinv_k must be >= 1");
    if (o.max_iters < 0 || o.bland_after < 0 || o.spin_timeout_cycles <= 0 || o.threads < 0 ||
        o.group_elems < 0 || o.device < 0 || o.device >= 64)
        return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: option out of range");
    for (int k = 0; k < count; ++k) {
        if (m[k] < 1 || n[k] < 1 || !A[k] || !b[k] || !c[k])
            return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: LP %d: bad size or NULL input", k);
        if (sense && sense[k] != LP_MAX_LE && sense[k] != LP_MIN_GE)
            return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: LP %d: unknown sense", k);
        if ((long long)n[k] + m[k] + 1 > 0x7fffffffll - 64)
            return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: LP %d too large", k);
    }
    DeviceRestore restore_;
    B_TRY(cudaSetDevice(o.device));
    int sms = 0;
    B_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device));
    // FP32 tableaus pivot with the FP64 reinversion between rounds of
    // reinv_k pivots; the pivot rule of an LP may switch, so its selection
    // scratch is sized for either rule
    const bool fp32 = o.precision == LP_FP32_REINV;
    const int prec = fp32 ? PREC_FP32 : PREC_FP64;
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    const int vw = fp32 ? 4 : 2, sector = fp32 ? 8 : 4;
    int threads = o.threads > 0 ? std::min(o.threads, 512) : 512;
    threads = std::max(64, (threads + 31) / 32 * 32);
    const long long gelems = o.group_elems > 0 ? o.group_elems : 262144;

    // shapes: CTAs per LP from its tableau size, strips of whole sectors
    std::vector<int> M(count), N(count), G(count), W(count), sv(count);
    std::vector<long long> P(count);
    size_t smem_max = 0, sprow_max = 0;
    for (int k = 0; k < count; ++k) {
        M[k] = m[k] + 1;
        N[k] = n[k] + m[k] + 1;
        P[k] = pitch_for(N[k]);
        sv[k] = sense ? sense[k] : 0;
        const long long gmin = (P[k] + (long long)threads * vw - 1) / ((long long)threads * vw);
        long long g = ((long long)M[k] * P[k] + gelems - 1) / gelems;
        g = std::min<long long>(g, std::min<long long>(sms, P[k] / sector));
        g = std::max<long long>(g, gmin);
        long long w = (P[k] + g - 1) / g;
        w = (w + sector - 1) / sector * sector;
        W[k] = (int)w;
        G[k] = (int)((P[k] + w - 1) / w);
        const size_t sprow = ((size_t)w * esz + 15) & ~(size_t)15;
        const size_t scol = ((size_t)M[k] * esz + 15) & ~(size_t)15;
        const size_t sr = (size_t)(sv[k] == 0 && !fp32 ? M[k] : N[k]) * sizeof(double);
        smem_max = std::max(smem_max, sprow + scol + sr);
        sprow_max = std::max(sprow_max, sprow);
    }
    const int use_smem = smem_max <= 200 * 1024 ? 1 : 0;
    const size_t smem = use_smem ? smem_max : sprow_max;
    const int ctas = max_coresident_batch_ctas(prec, threads, smem, use_smem, sms);
    const int max_group = *std::max_element(G.begin(), G.end());
    if (ctas < max_group)
        return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: %d co-resident CTAs, a group needs %d",
                     ctas, max_group);

    // work items, largest LPs first
    std::vector<int> order(count);
    for (int k = 0; k < count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b2) {
        return (long long)M[a] * P[a] > (long long)M[b2] * P[b2];
    });
    std::vector<int2> items;
    for (int k : order)
        for (int r = 0; r < G[k]; ++r) items.push_back(make_int2(k, r));

    // layout: meta block (mirrored in pinned memory) then the big arrays
    std::vector<long long> in_off(count), t_off(count), xy_off(count), scr_off(count);
    long long in_total = 0, xy_total = 0;
    size_t t_total = 0, scr_total = 0;
    for (int k = 0; k < count; ++k) {
        in_off[k] = in_total;
        in_total += (long long)m[k] * n[k] + m[k] + n[k];
        xy_off[k] = xy_total;
        xy_total += n[k] + m[k];
        t_off[k] = (long long)t_total;
        t_total += up256((size_t)M[k] * (size_t)P[k] * esz);
        scr_off[k] = (long long)scr_total;
        if (!use_smem) {
            const size_t scol = ((size_t)M[k] * esz + 15) & ~(size_t)15;
            const size_t sr = (size_t)(sv[k] == 0 && !fp32 ? M[k] : N[k]) * sizeof(double);
            scr_total += (size_t)G[k] * up256(scol + sr);
        }
    }
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off += up256(bytes); return at; };
    const size_t o_in_off = take(count * sizeof(long long)), o_t_off = take(count * sizeof(long long)),
                 o_xy_off = take(count * sizeof(long long)), o_m = take(count * sizeof(int)),
                 o_n = take(count * sizeof(int)), o_sense = take(count * sizeof(int)),
                 o_P = take(count * sizeof(long long)), o_bptr = take(count * sizeof(int *)),
                 o_items = take(items.size() * sizeof(int2)), o_src = take(3 * count * sizeof(double *)),
                 o_len = take(3 * count * sizeof(long long)), o_dst = take(3 * count * sizeof(long long)),
                 o_desc = take(count * sizeof(LpDesc));
    const size_t meta_bytes = off;
    size_t basis_total = 0, part_total = 0;
    for (int k = 0; k < count; ++k) {
        basis_total += up256((size_t)m[k] * sizeof(int));
        part_total += up256(2 * (size_t)G[k] * sizeof(Cand));
    }
    const size_t o_stats = take(count * sizeof(InputStats)), o_queue = take(sizeof(unsigned)),
                 o_obj = take(count * sizeof(double)), o_bar = take((size_t)count * 512),
                 o_basis = take(basis_total), o_part = take(part_total),
                 o_xy = take(xy_total * sizeof(double)), o_inp = take(in_total * sizeof(double)),
                 o_scr = take(scr_total), o_T = take(t_total);
    const size_t dev_total = off;
    const size_t pin_total = meta_bytes + up256(count * sizeof(InputStats)) +
                             up256(count * sizeof(double)) + up256(xy_total * sizeof(double)) +
                             up256(in_total * sizeof(double));

    Pool &pool = g_pool[o.device];
    std::lock_guard<std::mutex> lock(pool.mu);
    void *dv = nullptr, *pv = nullptr;
    B_TRY(pool_dev(pool, dev_total, &dv));
    B_TRY(pool_pin(pool, pin_total, &pv));
    unsigned char *D = static_cast<unsigned char *>(dv), *H = static_cast<unsigned char *>(pv);
    InputStats *h_stats = reinterpret_cast<InputStats *>(H + meta_bytes);
    double *h_obj = reinterpret_cast<double *>(H + meta_bytes + up256(count * sizeof(InputStats)));
    double *h_xy = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(h_obj) +
                                              up256(count * sizeof(double)));
    double *h_in = reinterpret_cast<double *>(reinterpret_cast<unsigned char *>(h_xy) +
                                              up256(xy_total * sizeof(double)));
    cudaStream_t s = (cudaStream_t)o.cuda_stream;

    // meta block
    memcpy(H + o_in_off, in_off.data(), count * sizeof(long long));
    memcpy(H + o_t_off, t_off.data(), count * sizeof(long long));
    memcpy(H + o_xy_off, xy_off.data(), count * sizeof(long long));
    memcpy(H + o_m, m, count * sizeof(int));
    memcpy(H + o_n, n, count * sizeof(int));
    memcpy(H + o_sense, sv.data(), count * sizeof(int));
    memcpy(H + o_P, P.data(), count * sizeof(long long));
    memcpy(H + o_items, items.data(), items.size() * sizeof(int2));
    {
        int **bp = reinterpret_cast<int **>(H + o_bptr);
        size_t bo = 0;
        for (int k = 0; k < count; ++k) {
            bp[k] = reinterpret_cast<int *>(D + o_basis + bo);
            bo += up256((size_t)m[k] * sizeof(int));
        }
    }
    cudaPointerAttributes pa;
    const bool dev_in = cudaPointerGetAttributes(&pa, A[0]) == cudaSuccess &&
                        (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev_in) {
        const double **src = reinterpret_cast<const double **>(H + o_src);
        long long *len = reinterpret_cast<long long *>(H + o_len);
        long long *dst = reinterpret_cast<long long *>(H + o_dst);
        for (int k = 0; k < count; ++k) {
            src[3 * k] = A[k];
            src[3 * k + 1] = b[k];
            src[3 * k + 2] = c[k];
            len[3 * k] = (long long)m[k] * n[k];
            len[3 * k + 1] = m[k];
            len[3 * k + 2] = n[k];
            dst[3 * k] = in_off[k];
            dst[3 * k + 1] = in_off[k] + len[3 * k];
            dst[3 * k + 2] = dst[3 * k + 1] + m[k];
        }
    }
    BatchArrays ba;
    ba.in_off = reinterpret_cast<const long long *>(D + o_in_off);
    ba.t_off = reinterpret_cast<const long long *>(D + o_t_off);
    ba.xy_off = reinterpret_cast<const long long *>(D + o_xy_off);
    ba.m = reinterpret_cast<const int *>(D + o_m);
    ba.n = reinterpret_cast<const int *>(D + o_n);
    ba.sense = reinterpret_cast<const int *>(D + o_sense);
    ba.P = reinterpret_cast<const long long *>(D + o_P);
    double *d_in = reinterpret_cast<double *>(D + o_inp);
    B_TRY(cudaMemcpyAsync(D, H, o_desc, cudaMemcpyHostToDevice, s));  // meta except descriptors
    if (dev_in) {
        batch_gather_kernel<<<dim3(16, 3 * count), 256, 0, s>>>(
            reinterpret_cast<const double *const *>(D + o_src),
            reinterpret_cast<const long long *>(D + o_dst),
            reinterpret_cast<const long long *>(D + o_len), d_in);
    } else {
        for (int k = 0; k < count; ++k) {
            double *p = h_in + in_off[k];
            memcpy(p, A[k], sizeof(double) * (size_t)m[k] * n[k]);
            memcpy(p + (size_t)m[k] * n[k], b[k], sizeof(double) * m[k]);
            memcpy(p + (size_t)m[k] * n[k] + m[k], c[k], sizeof(double) * n[k]);
        }
        B_TRY(cudaMemcpyAsync(d_in, h_in, in_total * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    InputStats *d_stats = reinterpret_cast<InputStats *>(D + o_stats);
    B_TRY(cudaMemsetAsync(d_stats, 0, count * sizeof(InputStats), s));
    batch_inspect_kernel<<<dim3(8, count), 256, 0, s>>>(ba, d_in, d_stats);
    B_TRY(cudaGetLastError());
    B_TRY(cudaMemcpyAsync(h_stats, d_stats, count * sizeof(InputStats), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));

    LpDesc *h_desc = reinterpret_cast<LpDesc *>(H + o_desc);
    size_t bo = 0, po = 0;
    for (int k = 0; k < count; ++k) {
        const InputStats &st = h_stats[k];
        if (st.flags & 4)
            return bfail(LP_ERR_INVALID_ARG, "lp_solve_batch: LP %d holds a NaN or infinity", k);
        if (sv[k] == LP_MAX_LE && (st.flags & 1))
            return bfail(LP_ERR_INFEASIBLE_START, "lp_solve_batch: LP %d: max form needs b >= 0", k);
        if (sv[k] == LP_MIN_GE && (st.flags & 2))
            return bfail(LP_ERR_INFEASIBLE_START, "lp_solve_batch: LP %d: min form needs c >= 0", k);
        double amax, bmax, cmax;
        memcpy(&amax, &st.amax_bits, 8);
        memcpy(&bmax, &st.bmax_bits, 8);
        memcpy(&cmax, &st.cmax_bits, 8);
        LpDesc d{};
        d.T = D + o_T + t_off[k];
        d.basis = reinterpret_cast<int *>(D + o_basis + bo);
        d.scratch = use_smem ? nullptr : D + o_scr + scr_off[k];
        if (!use_smem) {
            const size_t scol = ((size_t)M[k] * esz + 15) & ~(size_t)15;
            const size_t sr = (size_t)(sv[k] == 0 && !fp32 ? M[k] : N[k]) * sizeof(double);
            d.scratch_stride = (long long)up256(scol + sr);
        }
        d.part_sel = reinterpret_cast<Cand *>(D + o_part + po);
        d.bar = reinterpret_cast<unsigned *>(D + o_bar + (size_t)k * 512);
        d.err = reinterpret_cast<int *>(d.bar + 96);
        d.P = P[k];
        d.m = m[k];
        d.n = n[k];
        d.M = M[k];
        d.N = N[k];
        d.sense = sv[k];
        d.bland_after = o.bland_after;
        d.eps_d = o.eps_d > 0 ? o.eps_d : 1e-9 * std::max(1.0, cmax);
        d.eps_p = o.eps_p > 0 ? o.eps_p : 1e-9 * std::max(1.0, amax);
        d.eps_r = o.eps_r > 0 ? o.eps_r : 1e-9 * std::max(1.0, bmax);
        d.status = -1;
        d.last_p = d.last_q = -1;
        d.group = G[k];
        d.strip = W[k];
        h_desc[k] = d;
        bo += up256((size_t)m[k] * sizeof(int));
        po += up256(2 * (size_t)G[k] * sizeof(Cand));
    }
    LpDesc *d_desc = reinterpret_cast<LpDesc *>(D + o_desc);
    B_TRY(cudaMemcpyAsync(d_desc, h_desc, count * sizeof(LpDesc), cudaMemcpyHostToDevice, s));
    B_TRY(cudaMemsetAsync(D + o_bar, 0, (size_t)count * 512, s));
    B_TRY(cudaMemsetAsync(D + o_queue, 0, sizeof(unsigned), s));
    if (fp32)
        batch_build_kernel<float><<<dim3(16, count), 256, 0, s>>>(
            ba, d_in, D + o_T, reinterpret_cast<int *const *>(D + o_bptr));
    else
        batch_build_kernel<double><<<dim3(16, count), 256, 0, s>>>(
            ba, d_in, D + o_T, reinterpret_cast<int *const *>(D + o_bptr));
    B_TRY(cudaGetLastError());
    double *d_xy = reinterpret_cast<double *>(D + o_xy), *d_obj = reinterpret_cast<double *>(D + o_obj);
    if (fp32) {
        BatchFp32 f;
        f.count = count;
        f.m = m;
        f.n = n;
        f.sv = sv.data();
        f.G = G.data();
        f.order = order.data();
        f.in_off = in_off.data();
        f.t_off = t_off.data();
        f.xy_off = xy_off.data();
        f.P = P.data();
        f.d_in = d_in;
        f.d_T = D + o_T;
        f.d_xy = d_xy;
        f.d_obj = d_obj;
        f.h_desc = h_desc;
        f.d_desc = reinterpret_cast<LpDesc *>(D + o_desc);
        f.h_items = reinterpret_cast<int2 *>(H + o_items);
        f.d_items = reinterpret_cast<int2 *>(D + o_items);
        f.d_queue = reinterpret_cast<unsigned *>(D + o_queue);
        f.d_bar = D + o_bar;
        f.ctas = ctas;
        f.threads = threads;
        f.smem = smem;
        f.use_smem = use_smem;
        f.sms = sms;
        f.opt = &o;
        f.s = s;
        lp_status *fin = nullptr;
        double kms = 0.0;
        std::vector<lp_status> fstat(count, LP_NOT_SOLVED);
        fin = fstat.data();
        const lp_err fe = solve_batch_fp32(f, fin, &kms);
        if (fe != LP_OK) return fe;
        B_TRY(cudaMemcpyAsync(h_obj, d_obj, count * sizeof(double), cudaMemcpyDeviceToHost, s));
        if (x || y)
            B_TRY(cudaMemcpyAsync(h_xy, d_xy, xy_total * sizeof(double), cudaMemcpyDeviceToHost, s));
        B_TRY(cudaStreamSynchronize(s));
        long long piv = 0;
        for (int k = 0; k < count; ++k) {
            if (obj) obj[k] = h_obj[k];
            if (status) status[k] = fin[k];
            if (iters) iters[k] = h_desc[k].iters;
            piv += h_desc[k].iters;
            if (x && x[k]) memcpy(x[k], h_xy + xy_off[k], sizeof(double) * n[k]);
            if (y && y[k]) memcpy(y[k], h_xy + xy_off[k] + n[k], sizeof(double) * m[k]);
        }
        std::lock_guard<std::mutex> sl(g_stats_mu);
        g_last.kernel_ms = kms;
        g_last.pivots = piv;
        g_last.ctas = ctas;
        g_last.threads = threads;
        g_last.items = (int)items.size();
        g_last.max_group = max_group;
        return LP_OK;
    }
    cudaEvent_t e0, e1;
    B_TRY(cudaEventCreate(&e0));
    B_TRY(cudaEventCreate(&e1));
    B_TRY(cudaEventRecord(e0, s));
    B_TRY(launch_batch(prec, d_desc, reinterpret_cast<const int2 *>(D + o_items), (int)items.size(),
                       reinterpret_cast<unsigned *>(D + o_queue), ctas, threads, smem, use_smem,
                       o.spin_timeout_cycles, o.max_iters, s));
    B_TRY(cudaEventRecord(e1, s));
    batch_extract_kernel<double><<<count, 256, 0, s>>>(ba, D + o_T,
                                                       reinterpret_cast<int *const *>(D + o_bptr),
                                                       d_xy, d_obj);
    B_TRY(cudaGetLastError());
    B_TRY(cudaMemcpyAsync(h_desc, d_desc, count * sizeof(LpDesc), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaMemcpyAsync(h_obj, d_obj, count * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (x || y)
        B_TRY(cudaMemcpyAsync(h_xy, d_xy, xy_total * sizeof(double), cudaMemcpyDeviceToHost, s));
    B_TRY(cudaStreamSynchronize(s));
    float kms = 0.0f;
    cudaEventElapsedTime(&kms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    long long piv = 0;
    for (int k = 0; k < count; ++k) {
        if (obj) obj[k] = h_obj[k];
        if (status) status[k] = (lp_status)h_desc[k].status;
        if (iters) iters[k] = h_desc[k].iters;
        piv += h_desc[k].iters;
        if (x && x[k]) memcpy(x[k], h_xy + xy_off[k], sizeof(double) * n[k]);
        if (y && y[k]) memcpy(y[k], h_xy + xy_off[k] + n[k], sizeof(double) * m[k]);
    }
    {
        std::lock_guard<std::mutex> sl(g_stats_mu);
        g_last.kernel_ms = kms;
        g_last.pivots = piv;
        g_last.ctas = ctas;
        g_last.threads = threads;
        g_last.items = (int)items.size();
        g_last.max_group = max_group;
    }
    return LP_OK;
}

extern "C" lp_err lp_batch_stats(double *kernel_ms, long long *pivots, int *ctas, int *threads,
                                 int *max_group) {
    std::lock_guard<std::mutex> sl(g_stats_mu);
    if (kernel_ms) *kernel_ms = g_last.kernel_ms;
    if (pivots) *pivots = g_last.pivots;
    if (ctas) *ctas = g_last.ctas;
    if (threads) *threads = g_last.threads;
    if (max_group) *max_group = g_last.max_group;
    return LP_OK;
}

// ------------------------------------------------------------- autotuner --
//
// Picks the batched launch shape (tableau elements per CTA of a group, CTA
// size) for a batch by timing every candidate on the batch itself (the best
// of two solves each, batched pivot kernel time).  Results are cached in a
// text file, one line "key group_elems threads kernel_ms" per batch
// signature (count and a hash of the sorted shapes), so a serving process
// tunes once per workload mix.

namespace {

unsigned long long shape_signature(int count, const int *m, const int *n) {
    std::vector<unsigned long long> v(count);
    for (int k = 0; k < count; ++k) v[k] = ((unsigned long long)m[k] << 32) | (unsigned)n[k];
    std::sort(v.begin(), v.end());
    unsigned long long h = 1469598103934665603ull;  // FNV-1a
    for (unsigned long long x : v)
        for (int i = 0; i < 8; ++i) {
            h ^= (x >> (8 * i)) & 0xffu;
            h *= 1099511628211ull;
        }
    return h;
}

bool cache_lookup(const char *path, const char *key, long long *ge, int *th) {
    if (!path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[128];
    long long g;
    int t;
    double ms;
    bool hit = false;
    while (fscanf(f, "%127s %lld %d %lf", k, &g, &t, &ms) == 4)
        if (!strcmp(k, key)) {
            *ge = g;
            *th = t;
            hit = true;
        }
    fclose(f);
    return hit;
}

}  // namespace

extern "C" lp_err lp_batch_autotune(int count, const int *m, const int *n,
                                    const double *const *A, const double *const *b,
                                    const double *const *c, const int *sense,
                                    const lp_options *opt, const char *cache_path,
                                    lp_options *best) {
    if (!best) return bfail(LP_ERR_INVALID_ARG, "lp_batch_autotune: best is NULL");
    lp_options o;
    if (opt) o = *opt; else lp_options_default(&o);
    if (count < 1 || !m || !n) return bfail(LP_ERR_INVALID_ARG, "lp_batch_autotune: empty batch");
    char key[128];
    snprintf(key, sizeof key, "fp64-c%d-%016llx", count, shape_signature(count, m, n));
    long long ge = 0;
    int th = 0;
    if (cache_lookup(cache_path, key, &ge, &th)) {
        *best = o;
        best->group_elems = ge;
        best->threads = th;
        return LP_OK;
    }
    static const long long kElems[] = {16384, 65536, 262144, 1048576};
    static const int kThreads[] = {256, 512};
    double best_ms = 1e300;
    for (long long e : kElems)
        for (int t : kThreads) {
            lp_options trial = o;
            trial.group_elems = e;
            trial.threads = t;
            double ms = 1e300;
            for (int rep = 0; rep < 2; ++rep) {
                lp_err r = lp_solve_batch(count, m, n, A, b, c, sense, &trial, nullptr, nullptr,
                                          nullptr, nullptr, nullptr);
                if (r != LP_OK) return r;
                double k_ms = 0.0;
                lp_batch_stats(&k_ms, nullptr, nullptr, nullptr, nullptr);
                ms = std::min(ms, k_ms);
            }
            if (ms < best_ms) {
                best_ms = ms;
                ge = e;
                th = t;
            }
        }
    *best = o;
    best->group_elems = ge;
    best->threads = th;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (f) {
            fprintf(f, "%s %lld %d %.4f\n", key, ge, th, best_ms);
            fclose(f);
        }
    }
    return LP_OK;
}
