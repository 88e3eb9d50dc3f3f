// Dense tableau simplex kernels for sm_103a: the in-place kernel (one grid
// barrier per pivot; also run by batched and served solves), the batch and
// server kernels, and the build, inspection and extraction kernels.  The
// pipelined kernels are in gbs_pipe.cu.
//
// One persistent grid runs whole pivot sequences (the paper's Step I keeps its
// thread team alive for the whole solve, Sec. 3; here the team is a grid of
// CTAs, one per SM, that never returns to the host between pivots).
//
// Work split.  CTA g owns the column strip [g*W, g*W + W) of every row.  One
// pivot is one phase between two grid barriers:
//
//   1. Selection, computed redundantly by every CTA (no second barrier):
//      the per-CTA partials of the previous phase give the entering column q
//      (primal, Sec. 2 Step 2) or the leaving row r (dual simplex); then the
//      ratio test over all rows (primal, Step 3) or over all columns of row r
//      (dual), staging the pre-update pivot column in shared memory.  The
//      ratios are screened with a single-precision reciprocal and only the
//      rows within 2^-19 of the smallest screened ratio get the exact IEEE
//      division, so the selection equals the exact one.
//   2. Step 4 on the CTA's strip of the pivot row (IEEE division), into
//      shared memory.
//   3. Step 5 on the strip, T[i][j] = fma(-col[i], prow[j], T[i][j]) for every
//      row but the pivot row, objective row included, 128-bit vectors.  The
//      objective row (primal) or the rhs column (dual) is inspected as it is
//      written, giving this CTA's partial for the next selection -- the
//      paper's Step VI fuses the objective-row update with the next pricing
//      the same way.
//
// Race freedom.  A CTA writes only its own strip.  The data other CTAs read
// during selection -- primal: the pivot column and the rhs column; dual: the
// pivot column, row r and the objective row -- is written last: every CTA
// bumps a counter once its selection reads are done, and a strip's protected
// part is written only after the counter shows all CTAs arrived (by then it
// normally has, so this wait costs nothing).  Partials are double-buffered
// by pivot parity.
//
// Waits are bounded: a barrier or counter wait that does not complete within
// the spin limit sets the error flag and the kernel returns with status
// TIMEOUT.

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <stddef.h>
#include <stdint.h>
#include <utility>

#include "gbs_device.cuh"
#include "gbs_internal.h"

namespace gbs {

cudaError_t allow_dyn_smem(const void *fn) {
    static std::mutex mu;
    static std::map<std::pair<const void *, int>, int> limit;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int bytes;
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = limit.find({fn, dev});
        if (it != limit.end()) {
            bytes = it->second;
        } else {
            cudaFuncAttributes fa;
            int optin = 0;
            if ((e = cudaFuncGetAttributes(&fa, fn)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
                cudaSuccess)
                return e;
            bytes = optin - (int)fa.sharedSizeBytes;
            limit[{fn, dev}] = bytes;
        }
    }
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

namespace {

using namespace dev;


// Per-thread running candidate of the next selection, fed with freshly
// updated values: the objective row (primal pricing, Sec. 2 Step 2) or the
// rhs column (dual simplex leaving row).
struct Watch {
    unsigned long long lim_d, lim_r, zero;  // okey(-eps_d), okey(-eps_r), okey(0)
    int sense, m, N, bland, p, q;
    const int *basis;
};

template <typename T, typename V>
__device__ __forceinline__ void watch_row(Cand &best, const Watch &w, int i, int col0, const V &t,
                                          int rhs_lane) {
    constexpr int VW = Vec<T>::W;
    if (w.sense == 0) {
        if (i == w.m) {
#pragma unroll
            for (int k = 0; k < VW; ++k) {
                const int j = col0 + k;
                const unsigned long long zk = okey(getc(t, k));
                if (j < w.N - 1 && zk < w.lim_d) cand_take(best, w.bland ? w.zero : zk, j, j);
            }
        }
    } else if (rhs_lane >= 0 && i < w.m) {
        const unsigned long long vk = okey(getc(t, rhs_lane));
        if (vk < w.lim_r) {
            const int key = w.bland ? (i == w.p ? w.q : __ldcg(w.basis + i)) : i;
            cand_take(best, w.bland ? w.zero : vk, key, i);
        }
    }
}

// SMEM: the selection scratch lives in shared memory (else in this CTA's
// slice of global scratch); DUAL: dual simplex (else primal).  Template
// parameters, so that the update loop carries no per-row tests for them.
//
// solve_lp runs the pivots of one LP on a group of G co-resident CTAs (this
// CTA is rank g of the group); the group's barrier words, reader counter,
// partials and timeout flag live in the LP's descriptor.  The single-LP
// kernel below is one group spanning the grid; the batched kernel forms groups
// from a work queue.
template <typename T, bool SMEM, bool DUAL>
__device__ __forceinline__ void solve_lp(LpDesc *__restrict__ d, int G, int g, int W,
                                         long long spin_limit, long long budget,
                                         unsigned char *smem_raw) {
    typedef typename Vec<T>::type V;
    constexpr int VW = Vec<T>::W;
    constexpr int sense = DUAL ? 1 : 0;
    __shared__ Cand rbuf[4][32];
    __shared__ unsigned long long ubuf[32];
    __shared__ int s_flag;

    const int tid = threadIdx.x, B = blockDim.x;
    T *__restrict__ Tab = reinterpret_cast<T *>(d->T);
    int *__restrict__ basis = d->basis;
    const long long P = d->P;
    const int m = d->m, M = d->M, N = d->N;
    const int bland_after = d->bland_after;
    const unsigned long long lim_p = okey((T)d->eps_p);       // a_iq >  eps_p
    const unsigned long long lim_np = okey((T)(-d->eps_p));   // a_rj < -eps_p
    const unsigned long long zero_k = okey((T)0);
    long long iters = d->iters;
    const long long iter_limit =
        iters > 0x3fffffffffffffffll - budget ? 0x3fffffffffffffffll : iters + budget;
    int deg = d->deg;
    int status = ST_RUNNING;
    unsigned *readers = d->bar + 64;
    Watch w;
    w.lim_d = okey((T)(-d->eps_d));
    w.lim_r = okey((T)(-d->eps_r));
    w.zero = zero_k;
    w.sense = sense;
    w.m = m;
    w.N = N;
    w.basis = basis;

    // Per-CTA scratch: the strip of the normalised pivot row, the pre-update
    // pivot column and the screening keys (shared memory, or this CTA's slice
    // of a global scratch buffer when they do not fit).
    const size_t sprow_bytes = ((size_t)W * sizeof(T) + 15) & ~(size_t)15;
    const size_t scol_bytes = ((size_t)M * sizeof(T) + 15) & ~(size_t)15;
    T *sprow = reinterpret_cast<T *>(smem_raw);
    T *scol;
    unsigned long long *sr;
    if (SMEM) {
        scol = reinterpret_cast<T *>(smem_raw + sprow_bytes);
        sr = reinterpret_cast<unsigned long long *>(smem_raw + sprow_bytes + scol_bytes);
    } else {
        unsigned char *base = reinterpret_cast<unsigned char *>(d->scratch) +
                              (size_t)g * (size_t)d->scratch_stride;
        scol = reinterpret_cast<T *>(base);
        sr = reinterpret_cast<unsigned long long *>(base + scol_bytes);
    }

    // Column strip of this CTA and the thread -> (row lane, vector) map.
    const int c0 = g * W;  // < P: the host launches ceil(P / W) CTAs
    const int c1 = (int)min((long long)c0 + W, P);
    const int vpr = (c1 - c0) / VW;
    const int rpp = B / vpr;  // >= 1: the host keeps W <= B * VW
    const int lr = tid / vpr;
    const int lv = tid - lr * vpr;
    const bool active = lr < rpp;
    const int col0 = c0 + lv * VW;
    // the vector of this strip holding the rhs column, or -1
    const int rv = (N - 1 >= c0 && N - 1 < c1) ? (N - 1 - c0) / VW : -1;

    // Selection partials of the current tableau (parity buffer 0).
    {
        const int bland = deg >= bland_after;
        Cand c = cand_empty();
        if (!DUAL) {
            const T *z = Tab + (long long)m * P;
            for (int j = c0 + tid; j < c1 && j < N - 1; j += B) {
                const unsigned long long zk = okey(lds(z + j));
                if (zk < w.lim_d) cand_take(c, bland ? zero_k : zk, j, j);
            }
        } else if (rv >= 0) {
            for (int i = tid; i < m; i += B) {
                const unsigned long long vk = okey(lds(Tab + (long long)i * P + (N - 1)));
                if (vk < w.lim_r) cand_take(c, bland ? zero_k : vk, bland ? __ldcg(basis + i) : i, i);
            }
        }
        c = block_min_c(c, rbuf[3]);
        if (tid == 0) d->part_sel[g] = c;
    }
    if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) status = ST_TIMEOUT;

    unsigned rd_target = 0;
    int lk = 0;  // pivots made in this launch: selects the partials' parity buffer
    while (status == ST_RUNNING) {
        const int ab = tid == 0 ? abort_peek(d->abort) : 0;  // used at the pivot's barrier
        // ------------- selection, computed redundantly by every CTA -------------
        const int bland = deg >= bland_after;
        const Cand sel = load_partials_min(d->part_sel + (lk & 1) * G, G, rbuf[0]);
        if (sel.idx < 0) {
            status = ST_OPTIMAL;
            break;
        }
        if (iters >= iter_limit) {
            status = ST_ITER_LIMIT;
            break;
        }
        int p, q;
        unsigned long long rmin;
        if (!DUAL) {
            // Sec. 2 Step 3 over all rows: stage the pivot column, screen.
            q = sel.idx;
            unsigned long long lmin = ~0ull;
            for (int i = tid; i < M; i += B) {
                const T a = lds(Tab + (long long)i * P + q);
                const T rhs = lds(Tab + (long long)i * P + (N - 1));
                scol[i] = a;
                if (i < m) {
                    const unsigned long long rk = okey(a) > lim_p ? screen_key(pos_part(rhs), a) : ~0ull;
                    sr[i] = rk;
                    lmin = rk < lmin ? rk : lmin;
                }
            }
            const unsigned long long rstar = block_min_u(lmin, ubuf);
            if (rstar == ~0ull) {
                status = ST_UNBOUNDED;
                break;
            }
            const unsigned long long thr = screen_thr(rstar, (T)0);
            Cand c = cand_empty();
            for (int i = tid; i < m; i += B) {
                if (sr[i] <= thr) {
                    const T f = pos_part(lds(Tab + (long long)i * P + (N - 1))) / scol[i];
                    cand_take(c, okey(f), bland ? __ldcg(basis + i) : i, i);
                }
            }
            c = block_min_c(c, rbuf[1]);
            p = c.idx;
            rmin = c.vk;
        } else {
            // Dual simplex: leaving row from the partials, entering column by
            // the ratio over row r, then stage the pivot column.
            p = sel.idx;
            const T *rowr = Tab + (long long)p * P;
            const T *z = Tab + (long long)m * P;
            unsigned long long lmin = ~0ull;
            for (int j = tid; j < N - 1; j += B) {
                const T a = lds(rowr + j);
                const T zj = lds(z + j);
                const unsigned long long rk = okey(a) < lim_np ? screen_key(pos_part(zj), neg(a)) : ~0ull;
                sr[j] = rk;
                lmin = rk < lmin ? rk : lmin;
            }
            const unsigned long long rstar = block_min_u(lmin, ubuf);
            if (rstar == ~0ull) {
                status = ST_INFEASIBLE;
                break;
            }
            const unsigned long long thr = screen_thr(rstar, (T)0);
            Cand c = cand_empty();
            for (int j = tid; j < N - 1; j += B) {
                if (sr[j] <= thr) {
                    const T t = pos_part(lds(z + j)) / neg(lds(rowr + j));
                    cand_take(c, okey(t), j, j);
                }
            }
            c = block_min_c(c, rbuf[1]);
            q = c.idx;
            rmin = c.vk;
            for (int i = tid; i < M; i += B) scol[i] = lds(Tab + (long long)i * P + q);
        }
        // Every read of another CTA's columns for this pivot is done: arrive.
        __syncthreads();
        if (tid == 0) red_add_release(readers, 1u);
        rd_target += (unsigned)G;
        deg = (rmin == zero_k) ? deg + 1 : 0;
        w.bland = deg >= bland_after;  // rule of the next selection
        w.p = p;
        w.q = q;

        // ------------- Step 4: this CTA's strip of the pivot row -------------
        const T piv = scol[p];
        const T *rowp = Tab + (long long)p * P;
        for (int j = c0 + tid; j < c1; j += B) sprow[j - c0] = lds(rowp + j) / piv;
        __syncthreads();

        // ------------- Step 5, bulk of the strip -------------
        // Left for the pass below: the vector holding column q and the one
        // holding the rhs (other CTAs read them during selection; the rhs
        // vector also feeds the dual's next selection), the objective row
        // (it feeds the primal's next selection; the dual's selection reads
        // it) and, in the dual, row r.
        const int qv = (q >= c0 && q < c1) ? (q - c0) / VW : -1;
        if (active && lv != qv && lv != rv) {
            const V pr = *reinterpret_cast<const V *>(sprow + lv * VW);
            T *base = Tab + col0;
            int i = lr;
            for (; i + 3 * rpp < m; i += 4 * rpp) {
                const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                V *p0 = reinterpret_cast<V *>(base + (long long)i * P);
                V *p1 = reinterpret_cast<V *>(base + (long long)i1 * P);
                V *p2 = reinterpret_cast<V *>(base + (long long)i2 * P);
                V *p3 = reinterpret_cast<V *>(base + (long long)i3 * P);
                const V t0 = ldv(p0), t1 = ldv(p1), t2 = ldv(p2), t3 = ldv(p3);
                const T a0 = scol[i], a1 = scol[i1], a2 = scol[i2], a3 = scol[i3];
                const V u0 = pivot_vec<T>(t0, i, p, a0, pr);
                const V u1 = pivot_vec<T>(t1, i1, p, a1, pr);
                const V u2 = pivot_vec<T>(t2, i2, p, a2, pr);
                const V u3 = pivot_vec<T>(t3, i3, p, a3, pr);
                if (!DUAL || i != p) *p0 = u0;
                if (!DUAL || i1 != p) *p1 = u1;
                if (!DUAL || i2 != p) *p2 = u2;
                if (!DUAL || i3 != p) *p3 = u3;
            }
            for (; i < m; i += rpp) {
                if (DUAL && i == p) continue;
                V *p0 = reinterpret_cast<V *>(base + (long long)i * P);
                *p0 = pivot_vec<T>(ldv(p0), i, p, scol[i], pr);
            }
        }
        if (!wait_count(readers, rd_target, d->err, spin_limit, &s_flag)) {
            status = ST_TIMEOUT;
            break;
        }
        // ------------- Step 5, the rest, with the next selection's partials -----
        Cand watch = cand_empty();
        // (a) the q and rhs vectors, every row, spread over all threads
        for (int k = 0; k < 2; ++k) {
            const int v = k == 0 ? qv : (rv != qv ? rv : -1);
            if (v < 0) continue;
            const int vcol0 = c0 + v * VW;
            const int vrhs = (N - 1 >= vcol0 && N - 1 < vcol0 + VW) ? (N - 1 - vcol0) : -1;
            const V vpr_ = *reinterpret_cast<const V *>(sprow + v * VW);
            T *vbase = Tab + vcol0;
#pragma unroll 4
            for (int i = tid; i < M; i += B) {
                V *p0 = reinterpret_cast<V *>(vbase + (long long)i * P);
                const V u0 = pivot_vec<T>(ldv(p0), i, p, scol[i], vpr_);
                *p0 = u0;
                watch_row<T>(watch, w, i, vcol0, u0, vrhs);
            }
        }
        // (b) the objective row and, in the dual, row r, for the other vectors
        for (int k = tid; k < (DUAL ? 2 : 1) * vpr; k += B) {
            const int v = k % vpr;
            if (v == qv || v == rv) continue;
            const int i = k < vpr ? m : p;
            const int vcol0 = c0 + v * VW;
            V *p0 = reinterpret_cast<V *>(Tab + vcol0 + (long long)i * P);
            const V u0 = pivot_vec<T>(ldv(p0), i, p, scol[i],
                                      *reinterpret_cast<const V *>(sprow + v * VW));
            *p0 = u0;
            watch_row<T>(watch, w, i, vcol0, u0, -1);
        }
        if (g == 0 && tid == 0) {
            if (iters < d->trace_cap) {
                d->trace[2 * iters] = p;
                d->trace[2 * iters + 1] = q;
            }
            basis[p] = q;
            d->last_p = p;
            d->last_q = q;
        }
        watch = block_min_c(watch, rbuf[2]);
        if (tid == 0) d->part_sel[((lk + 1) & 1) * G + g] = watch;
        // past the host's deadline: the flag ends every CTA's barrier below
        if (ab) atomicExch(d->err, 1);
        ++iters;
        ++lk;
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

template <typename T, bool SMEM, bool DUAL>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pivot_kernel(LpDesc *__restrict__ d, int W, long long spin_limit, long long budget) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_lp<T, SMEM, DUAL>(d, gridDim.x, blockIdx.x, W, spin_limit, budget, smem_raw);
}

constexpr int kBatchThreads = 512;  // register room for both pivot rules in one kernel

// ---------------------------------------------------------------------------
// Serving: continuous batching in one persistent kernel.
//
// CTA 0 dispatches: it reads the slots the host made ready from a ring in
// mapped host memory and publishes, for each, `group` consecutive work items
// (slot, rank) into a device ring.  The other CTAs are workers: each takes a
// ticket, waits until the item of that ticket is published, and runs that
// rank of the slot's group; the group computes the input statistics and
// tolerances, builds the tableau (Sec. 2 Step 1), pivots with the same code
// as every other path, reads the solution off and marks the slot done in the
// host ring.  Requests that arrive while others are on the GPU are dispatched
// as soon as the host has a slot and memory for them, so their pivots overlap
// with the ones in flight.  When nothing arrives for idle_limit cycles and no
// slot is in flight, the dispatcher hands every worker an exit item and the
// kernel ends; the host relaunches it on the next request.  While busy but
// without new requests it hands waiting workers no-op items every idle_limit/2
// cycles, so no worker's bounded wait runs out during a long solve.

__device__ __forceinline__ int ld_acq_sys(const int *p) {
    int v;
    asm volatile("ld.acquire.sys.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_sys(int *p, int v) {
    asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ void serve_dispatch(ServeSlot *slots, ServeCtl *ctl, ServeRing *ring, int workers,
                               long long idle_limit) {
    if (threadIdx.x != 0) return;
    const long long keepalive = idle_limit / 2;
    long long idle0 = clock64(), alive0 = idle0;
    unsigned tail = ctl->tail;
    auto publish = [&](int slot, int rank) {
        ctl->items[tail % kServeQueue] = make_int2(slot, rank);
        __threadfence();
        st_release(&ctl->seq[tail % kServeQueue], tail + 1u);
        ++tail;
    };
    for (;;) {
        const int rq_tail = ld_acq_sys(&ring->rq_tail);
        int rq_head = *(volatile int *)&ring->rq_head;
        bool any = false;
        while (rq_head != rq_tail) {
            const int s = *(volatile int *)&ring->rq[rq_head % kServeMaxSlots];
            const int G = *(volatile int *)&slots[s].d.group;
            atomicAdd(&ctl->in_flight, 1);
            for (int r = 0; r < G; ++r) publish(s, r);
            ++rq_head;
            st_rel_sys(&ring->rq_head, rq_head);
            any = true;
        }
        const long long now = clock64();
        if (any) {
            idle0 = alive0 = now;
        } else if (*(volatile int *)&ctl->err ||
                   (*(volatile int *)&ctl->in_flight == 0 &&
                    (ld_acq_sys(&ring->shutdown) || now - idle0 > idle_limit))) {
            break;
        } else {
            if (now - alive0 > keepalive) {
                // hand every worker waiting on a ticket a no-op item, which
                // restarts its bounded wait
                const unsigned head = *(volatile unsigned *)&ctl->head;
                while ((int)(head - tail) > 0) publish(-2, 0);
                alive0 = now;
            }
            __nanosleep(200);
        }
    }
    for (int k = 0; k < workers; ++k) publish(-1, 0);
    ctl->tail = tail;
}

__device__ __forceinline__ double block_max_dev(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double r = red[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); ++k) r = fmax(r, red[k]);
    return r;
}

__device__ void serve_slot(ServeSlot *S, int slot, int rank, ServeCtl *ctl, ServeRing *ring,
                           long long spin_limit, unsigned char *smem_raw) {
    __shared__ double red[32];
    __shared__ int s_flag, s_fl;
    LpDesc *d = &S->d;
    const int G = d->group, m = d->m, n = d->n, M = d->M, N = d->N, tid = threadIdx.x,
              B = blockDim.x;
    const long long P = d->P;
    const int sense = d->sense;
    // input statistics over this rank's slice
    {
        double amax = 0.0, bmax = 0.0, cmax = 0.0;
        int fl = 0;
        const long long L = (long long)m * n;
        const long long a0 = L * rank / G, a1 = L * (rank + 1) / G;
        for (long long e = a0 + tid; e < a1; e += B) {
            const double v = S->A[e];
            if (!isfinite(v)) fl |= 4; else amax = fmax(amax, fabs(v));
        }
        for (int i = (int)((long long)m * rank / G) + tid; i < (int)((long long)m * (rank + 1) / G); i += B) {
            const double v = S->b[i];
            if (!isfinite(v)) fl |= 4; else bmax = fmax(bmax, fabs(v));
            if (v < 0.0) fl |= 1;
        }
        for (int j = (int)((long long)n * rank / G) + tid; j < (int)((long long)n * (rank + 1) / G); j += B) {
            const double v = S->c[j];
            if (!isfinite(v)) fl |= 4; else cmax = fmax(cmax, fabs(v));
            if (v < 0.0) fl |= 2;
        }
        if (tid == 0) s_fl = 0;
        __syncthreads();
        if (fl) atomicOr(&s_fl, fl);
        amax = block_max_dev(amax, red);
        bmax = block_max_dev(bmax, red);
        cmax = block_max_dev(cmax, red);
        if (tid == 0) {
            if (amax > 0.0) atomicMax(&S->stats->amax_bits, (unsigned long long)__double_as_longlong(amax));
            if (bmax > 0.0) atomicMax(&S->stats->bmax_bits, (unsigned long long)__double_as_longlong(bmax));
            if (cmax > 0.0) atomicMax(&S->stats->cmax_bits, (unsigned long long)__double_as_longlong(cmax));
            if (s_fl) atomicOr(&S->stats->flags, s_fl);
        }
    }
    bool ok = grid_sync(d->bar, d->err, G, spin_limit, &s_flag);
    const int flags = __ldcg(&S->stats->flags);
    const bool bad = (flags & 4) || (sense == 0 && (flags & 1)) || (sense == 1 && (flags & 2));
    if (rank == 0 && tid == 0) {
        const double amax = __longlong_as_double((long long)__ldcg(&S->stats->amax_bits));
        const double bmax = __longlong_as_double((long long)__ldcg(&S->stats->bmax_bits));
        const double cmax = __longlong_as_double((long long)__ldcg(&S->stats->cmax_bits));
        d->eps_d = S->opt_eps_d > 0 ? S->opt_eps_d : 1e-9 * fmax(1.0, cmax);
        d->eps_p = S->opt_eps_p > 0 ? S->opt_eps_p : 1e-9 * fmax(1.0, amax);
        d->eps_r = S->opt_eps_r > 0 ? S->opt_eps_r : 1e-9 * fmax(1.0, bmax);
    }
    // Sec. 2 Step 1 on this rank's rows
    if (ok && !bad) {
        const double sg = sense == 0 ? 1.0 : -1.0;
        double *Tab = reinterpret_cast<double *>(d->T);
        const long long e0 = (long long)M * P * rank / G, e1 = (long long)M * P * (rank + 1) / G;
        for (long long e = e0 + tid; e < e1; e += B) {
            const int i = (int)(e / P);
            const int j = (int)(e - (long long)i * P);
            double v = 0.0;
            if (i < m) {
                if (j < n) v = sg * S->A[(long long)i * n + j];
                else if (j == n + i) v = 1.0;
                else if (j == N - 1) v = sg * S->b[i];
            } else if (j < n) {
                v = -sg * S->c[j];
            }
            Tab[e] = v;
        }
        for (int i = (int)((long long)m * rank / G) + tid; i < (int)((long long)m * (rank + 1) / G); i += B)
            d->basis[i] = n + i;
    }
    if (ok) ok = grid_sync(d->bar, d->err, G, spin_limit, &s_flag);
    if (ok && !bad) {
        if (sense)
            solve_lp<double, true, true>(d, G, rank, d->strip, spin_limit, S->budget, smem_raw);
        else
            solve_lp<double, true, false>(d, G, rank, d->strip, spin_limit, S->budget, smem_raw);
    }
    if (rank != 0) return;
    __syncthreads();
    if (!ok || *(volatile int *)d->err) {
        // a group wait ran out: report it and stop the server taking work
        if (tid == 0) {
            d->status = ST_TIMEOUT;
            atomicExch(&ctl->err, 1);
        }
    } else if (bad) {
        if (tid == 0) d->status = (flags & 4) ? -2 : -3;  // invalid input / infeasible start
    } else {
        const double *Tab = reinterpret_cast<const double *>(d->T);
        const double *z = Tab + (long long)m * P;
        for (int j = tid; j < n; j += B) S->x[j] = 0.0;
        for (int i = tid; i < m; i += B) S->y[i] = __ldcg(z + n + i);
        __syncthreads();
        for (int i = tid; i < m; i += B) {
            const int j = __ldcg(d->basis + i);
            if (j < n) S->x[j] = __ldcg(Tab + (long long)i * P + (N - 1));
        }
        if (tid == 0) {
            const double zv = __ldcg(z + N - 1);
            *S->obj = sense == 0 ? zv : -zv;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence_system();
        atomicSub(&ctl->in_flight, 1);
        st_rel_sys(&ring->done[slot], 1);
    }
}

__global__ void __launch_bounds__(kBatchThreads)
    server_kernel(ServeSlot *slots, int nslots, ServeCtl *ctl, ServeRing *ring,
                  long long spin_limit, long long idle_limit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (blockIdx.x == 0) {
        serve_dispatch(slots, ctl, ring, gridDim.x - 1, idle_limit);
        return;
    }
    __shared__ int2 s_item;
    __shared__ int s_ok;
    const long long wait_limit = idle_limit + spin_limit;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const unsigned t = atomicAdd(&ctl->head, 1u);
            int ok = 1;
            const long long t0 = clock64();
            while (ld_acquire(&ctl->seq[t % kServeQueue]) != t + 1u) {
                if (clock64() - t0 > wait_limit) {
                    atomicExch(&ctl->err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(256);
            }
            s_ok = ok;
            if (ok) {
                s_item.x = __ldcg(&ctl->items[t % kServeQueue].x);
                s_item.y = __ldcg(&ctl->items[t % kServeQueue].y);
            }
        }
        __syncthreads();
        if (!s_ok || s_item.x == -1) break;
        if (s_item.x < 0) continue;  // keep-alive
        serve_slot(slots + s_item.x, s_item.x, s_item.y, ctl, ring, spin_limit, smem_raw);
    }
}

// Many LPs in one persistent launch.  items[] lists (lp, rank) pairs, the
// ranks of one LP consecutive, largest LPs first; CTAs pop items in order
// from *queue, and the d->group CTAs that pop the ranks of one LP solve it
// together.  A group waits only on CTAs that hold earlier items, whose groups
// are complete, so every group forms (the launch has at least max(group)
// co-resident CTAs); all waits are bounded anyway.
template <typename T, bool SMEM>
__global__ void __launch_bounds__(kBatchThreads)
    batch_kernel(LpDesc *__restrict__ descs, const int2 *__restrict__ items, int nitems,
                 unsigned *queue, long long spin_limit, long long budget) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int2 w = items[it];
        LpDesc *d = descs + w.x;
        if (d->sense)
            solve_lp<T, SMEM, true>(d, d->group, w.y, d->strip, spin_limit, budget, smem_raw);
        else
            solve_lp<T, SMEM, false>(d, d->group, w.y, d->strip, spin_limit, budget, smem_raw);
    }
}

// ---------------------------------------------------------------------------

__device__ __forceinline__ double block_max(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;  // valid in thread 0
}

// max |A|, max |b|, max |c| (as bit patterns of non-negative doubles, whose
// unsigned order is the numeric order), sign and finiteness flags.  One
// atomic per CTA and quantity.
__global__ void __launch_bounds__(256) inspect_kernel(const double *__restrict__ A,
                                                      const double *__restrict__ b,
                                                      const double *__restrict__ c, int m, int n,
                                                      InputStats *out) {
    __shared__ double red[32];
    __shared__ int sflags;
    const long long total = (long long)m * n;
    double amax = 0.0, bmax = 0.0, cmax = 0.0;
    int flags = 0;
    if (threadIdx.x == 0) sflags = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long k = t0; k < total; k += stride) {
        const double v = A[k];
        if (!isfinite(v)) flags |= 4;
        else amax = fmax(amax, fabs(v));
        if ((unsigned long long)__double_as_longlong(v) == 0x8000000000000000ull) flags |= 8;
    }
    for (long long k = t0; k < m; k += stride) {
        const double v = b[k];
        if (!isfinite(v)) flags |= 4;
        else bmax = fmax(bmax, fabs(v));
        if (v < 0.0) flags |= 1;
        if ((unsigned long long)__double_as_longlong(v) == 0x8000000000000000ull) flags |= 8;
    }
    for (long long k = t0; k < n; k += stride) {
        const double v = c[k];
        if (!isfinite(v)) flags |= 4;
        else cmax = fmax(cmax, fabs(v));
        if (v < 0.0) flags |= 2;
    }
    __syncthreads();
    if (flags) atomicOr(&sflags, flags);
    amax = block_max(amax, red);
    bmax = block_max(bmax, red);
    cmax = block_max(cmax, red);
    if (threadIdx.x == 0) {
        if (amax > 0.0) atomicMax(&out->amax_bits, (unsigned long long)__double_as_longlong(amax));
        if (bmax > 0.0) atomicMax(&out->bmax_bits, (unsigned long long)__double_as_longlong(bmax));
        if (cmax > 0.0) atomicMax(&out->cmax_bits, (unsigned long long)__double_as_longlong(cmax));
        if (sflags) atomicOr(&out->flags, sflags);
    }
}

// Sec. 2 Step 1: the initial tableau (rows [A | I | b], objective row
// [-c | 0 | 0]; dual form [-A | I | -b] and [c | 0 | 0]), padded with zeros
// to the pitch P.  sense 2 is Phase 1 of Phase I (not in the paper): the
// rows of the primal form with the objective row [max(-c, 0) | 0 | 0], whose
// slack basis is dual feasible although some b_i < 0.
template <typename T>
__global__ void build_kernel(const double *__restrict__ A, const double *__restrict__ b,
                             const double *__restrict__ c, int m, int n, int sense,
                             T *__restrict__ Tab, long long P, int *__restrict__ basis) {
    const int N = n + m + 1;
    const long long total = (long long)(m + 1) * P;
    const double sg = sense == 1 ? -1.0 : 1.0;
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
            v = sense == 2 ? (c[j] < 0.0 ? -c[j] : 0.0) : -sg * c[j];
        }
        Tab[k] = (T)v;
    }
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m; k += stride)
        basis[k] = n + (int)k;
}

// Phase I, the start of Phase 2: the objective row of max c'x in the basis
// Phase 1 ended with, z_j = -c_j + sum_i c_B(i) T[i][j] (c_j = 0 for slack
// columns; the rhs column gives the objective value), summed over the rows
// in increasing order with one fma per row whose basic variable is
// structural (slack-basic rows cost 0).  One thread per column; FP64.
__global__ void phase2_objective_kernel(const LpDesc *__restrict__ d, const double *__restrict__ c) {
    double *Tab = reinterpret_cast<double *>(d->T);  // the buffer Phase 1 left current
    const int m = d->m, n = d->n, N = d->N;
    const long long P = d->P;
    const int *basis = d->basis;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        double z = j < n ? -c[j] : 0.0;
        for (int i = 0; i < m; ++i) {
            const int bi = basis[i];
            if (bi < n) z = fma(c[bi], Tab[(long long)i * P + j], z);
        }
        Tab[(long long)m * P + j] = z;
    }
}

// Solution read-off, part 1: zero x, duals from the objective row, objective.
template <typename T>
__global__ void extract_kernel1(const LpDesc *__restrict__ d, const T *Tab, int m, int n,
                                long long P, int sense, double *x, double *y, double *obj) {
    if (d) Tab = reinterpret_cast<const T *>(d->T);  // the buffer the pivot kernel left current
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
__global__ void extract_kernel2(const LpDesc *__restrict__ d, const T *Tab,
                                const int *__restrict__ basis, int m, int n, long long P,
                                double *x) {
    if (d) Tab = reinterpret_cast<const T *>(d->T);
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
    const long long work = (long long)m * n / 8;  // ~8 elements per thread
    inspect_kernel<<<grid_for(work, 256), 256, 0, s>>>(A, b, c, m, n, out);
    return cudaGetLastError();
}

cudaError_t launch_phase2_objective(const LpDesc *d_desc, const double *c, int N, cudaStream_t s) {
    phase2_objective_kernel<<<(N + 255) / 256, 256, 0, s>>>(d_desc, c);
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

PivotShape choose_shape(int prec, int sense, int M, int N, long long P, int sms, int threads,
                        int ctas) {
    PivotShape sh;
    const int vw = prec == PREC_FP64 ? 2 : 4;       // elements per 16-byte vector
    const int sector = prec == PREC_FP64 ? 4 : 8;   // elements per 32-byte sector
    const size_t esz = prec == PREC_FP64 ? sizeof(double) : sizeof(float);
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
    sh.dual = sense;
    const size_t sprow = ((size_t)w * esz + 15) & ~(size_t)15;
    const size_t scol = ((size_t)M * esz + 15) & ~(size_t)15;
    const size_t sr = (size_t)(sense == 0 ? M : N) * sizeof(double);
    if (sprow + scol + sr <= kMaxDynSmem) {
        sh.use_smem = 1;
        sh.smem_bytes = sprow + scol + sr;
        sh.scratch_stride = 0;
    } else {
        sh.use_smem = 0;
        sh.smem_bytes = sprow;
        sh.scratch_stride = (long long)((scol + sr + 255) & ~(size_t)255);
    }
    return sh;
}

cudaError_t launch_pivot(int prec, LpDesc *d_desc, const PivotShape &sh, long long spin_limit,
                         long long budget, cudaStream_t s) {
    if (sh.pipe) return launch_pivot_pipe(prec, d_desc, sh, spin_limit, budget, s);
    int W = sh.strip;
    void *args[] = {&d_desc, &W, &spin_limit, &budget};
    const void *fn;
    if (prec == PREC_FP64) {
        if (sh.dual)
            fn = sh.use_smem ? (const void *)pivot_kernel<double, true, true>
                             : (const void *)pivot_kernel<double, false, true>;
        else
            fn = sh.use_smem ? (const void *)pivot_kernel<double, true, false>
                             : (const void *)pivot_kernel<double, false, false>;
    } else {
        if (sh.dual)
            fn = sh.use_smem ? (const void *)pivot_kernel<float, true, true>
                             : (const void *)pivot_kernel<float, false, true>;
        else
            fn = sh.use_smem ? (const void *)pivot_kernel<float, true, false>
                             : (const void *)pivot_kernel<float, false, false>;
    }
    if (sh.smem_bytes > 0) {  // static shared memory counts against the 48 KB default too
        cudaError_t e = allow_dyn_smem(fn);
        if (e != cudaSuccess) return e;
    }
    // A cooperative launch fails instead of running when the grid cannot be
    // co-resident, which the grid barrier needs.
    return cudaLaunchCooperativeKernel(fn, dim3(sh.ctas), dim3(sh.threads), args, sh.smem_bytes, s);
}

cudaError_t launch_server(ServeSlot *slots, int nslots, ServeCtl *ctl, ServeRing *ring_dev,
                          int ctas, int threads, size_t smem, long long spin_limit,
                          long long idle_limit, cudaStream_t s) {
    void *args[] = {&slots, &nslots, &ctl, &ring_dev, &spin_limit, &idle_limit};
    const void *fn = (const void *)server_kernel;
    if (smem > 0) {  // static shared memory counts against the 48 KB default too
        cudaError_t e = allow_dyn_smem(fn);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(threads), args, smem, s);
}

int max_coresident_server_ctas(int threads, size_t smem, int sms) {
    const void *fn = (const void *)server_kernel;
    if (smem > 0) allow_dyn_smem(fn);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t launch_batch(int prec, LpDesc *descs, const int2 *items, int nitems, unsigned *queue,
                         int ctas, int threads, size_t smem, int use_smem, long long spin_limit,
                         long long budget, cudaStream_t s) {
    void *args[] = {&descs, &items, &nitems, &queue, &spin_limit, &budget};
    const void *fn;
    if (prec == PREC_FP64)
        fn = use_smem ? (const void *)batch_kernel<double, true> : (const void *)batch_kernel<double, false>;
    else
        fn = use_smem ? (const void *)batch_kernel<float, true> : (const void *)batch_kernel<float, false>;
    if (smem > 0) {  // static shared memory counts against the 48 KB default too
        cudaError_t e = allow_dyn_smem(fn);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(ctas), dim3(threads), args, smem, s);
}

int max_coresident_batch_ctas(int prec, int threads, size_t smem, int use_smem, int sms) {
    const void *fn;
    if (prec == PREC_FP64)
        fn = use_smem ? (const void *)batch_kernel<double, true> : (const void *)batch_kernel<double, false>;
    else
        fn = use_smem ? (const void *)batch_kernel<float, true> : (const void *)batch_kernel<float, false>;
    if (smem > 0) allow_dyn_smem(fn);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

cudaError_t launch_extract(int prec, const LpDesc *d_desc, const void *T, const int *basis,
                           int m, int n, long long P, int sense, double *x, double *y,
                           double *obj, cudaStream_t s) {
    const long long work = (long long)(m > n ? m : n);
    if (prec == PREC_FP64) {
        extract_kernel1<double><<<grid_for(work, 256), 256, 0, s>>>(
            d_desc, (const double *)T, m, n, P, sense, x, y, obj);
        extract_kernel2<double><<<grid_for(m, 256), 256, 0, s>>>(d_desc, (const double *)T,
                                                                 basis, m, n, P, x);
    } else {
        extract_kernel1<float><<<grid_for(work, 256), 256, 0, s>>>(
            d_desc, (const float *)T, m, n, P, sense, x, y, obj);
        extract_kernel2<float><<<grid_for(m, 256), 256, 0, s>>>(d_desc, (const float *)T, basis,
                                                                m, n, P, x);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_fp64(const float *T, long long P, int M, int N, double *out,
                           cudaStream_t s) {
    to_fp64_kernel<<<grid_for((long long)M * N, 256), 256, 0, s>>>(T, P, M, N, out);
    return cudaGetLastError();
}

}  // namespace gbs
