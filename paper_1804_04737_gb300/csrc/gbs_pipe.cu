// Pipelined simplex kernels for sm_103a: the next pivot's selection runs while
// the current pivot's update streams, in every CTA of one persistent grid.
//
//   pivot_pipe_kernel        primal, one pivot per pass, in place (tableaus
//                            that fit L2) or double-buffered
//   pivot_pipe_dual_kernel   dual simplex, one pivot per pass, double-buffered
//   pivot_block_kernel       primal, two pivots per pass, double-buffered
//   pivot_block_dual_kernel  dual simplex, two pivots per pass, double-buffered
//
// Every kernel applies the arithmetic of Sec. 2 Steps 2-5 in the one-pivot
// order (IEEE division for the pivot row, one fma per element and pivot), so
// pivots and results are bit for bit those of the in-place kernel
// (gbs_pivot.cu) and of the FP64 reference.  CTA g owns the column strip
// [g*W, g*W + W) of every row; a few warps per CTA select, the rest update.
// Waits are bounded: one that does not complete within the spin limit sets
// the error flag and the kernel returns with status TIMEOUT.

#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <stddef.h>
#include <stdint.h>

#include "gbs_device.cuh"
#include "gbs_internal.h"

namespace gbs {

namespace {

using namespace dev;

// ---------------------------------------------------------------------------
// Pipelined primal simplex for one LP (FP64 or FP32 tableau).
//
// In every CTA the last SW warps select pivot k+1 while the others
// stream pivot k's update of the CTA's column strip:
//   update warps     divide the strip of the pivot row (Step 4), update the
//                    strip of the objective row and publish the CTA's pricing
//                    record (its best column, with the new pivot-row values at
//                    that column and at the rhs), then update the rest of the
//                    strip (Step 5), reading the pivot column from this CTA's
//                    scratch;
//   selection warps  reduce the pricing records to the entering column q'
//                    (Step 2), form the whole column q' and rhs of tableau k+1
//                    with the very fma the update uses (so the values are bit
//                    for bit those the update writes) into the CTA's scratch,
//                    and run the screened ratio test on them (Step 3).  Every
//                    CTA does this redundantly, so the pivot row needs no
//                    exchange between CTAs.  The column comes from tableau k;
//                    the rhs from the CTA's own copy of the rhs column, which
//                    it carries in scratch from pivot to pivot.
// In place (tableaus that fit L2), the vector the selection reads (each CTA's
// own pricing winner, which is where the entering column always is) is left
// out of the bulk update and updated once a counter shows every CTA's
// selection done reading it.  There is no grid barrier: a CTA publishes its
// pricing record only after finishing its previous pivot, so the pricing
// counter also proves every vector the selection reads is current,
// and no CTA runs more than one pivot ahead of another (records are
// double-buffered by pivot parity).  Double-buffered (larger tableaus), pivot
// k reads one buffer and writes the other, with a grid barrier per pivot to
// keep the CTAs' row streams in step.  The selection divides only on
// near-ties: it shares the FP64 pipe with the update warps.  The first pivot's
// selection runs alone, with a grid barrier.

// Selection warps per CTA: four in place (the selection is the critical path
// of an L2-resident pivot), two double-buffered (the update is, and wants
// the warps); the two-pivot kernel takes four or eight.  kSelThreadsMax sizes
// the launch shape for any of them.
constexpr int kSelThreadsMax = 256;
constexpr int kSelRows = 4;  // rows in flight per selection thread, two loads each
constexpr int kColRows = 8;  // the same with one load per row

__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }

__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

static_assert(sizeof(Cand) == 16 && offsetof(Cand, key) == 8 && offsetof(Cand, idx) == 12,
              "Cand is read as one 16-byte vector");

__device__ __forceinline__ unsigned long long tbits(double x) {
    return (unsigned long long)__double_as_longlong(x);
}
__device__ __forceinline__ unsigned long long tbits(float x) {
    return (unsigned long long)__float_as_uint(x);
}
template <typename T>
__device__ __forceinline__ T tfrom(unsigned long long u);
template <>
__device__ __forceinline__ double tfrom<double>(unsigned long long u) {
    return __longlong_as_double((long long)u);
}
template <>
__device__ __forceinline__ float tfrom<float>(unsigned long long u) {
    return __uint_as_float((unsigned)u);
}

__device__ __forceinline__ Cand unpack_cand(const ulonglong2 &v) {
    Cand e;
    e.vk = v.x;
    e.key = (int)(unsigned)(v.y & 0xffffffffull);
    e.idx = (int)(unsigned)(v.y >> 32);
    return e;
}

// This selection thread's minimum over the G records stid, stid + NT, ...,
// with a tag of its winner: vals[k].x when vals is given, else the record
// index k.  The records of one thread are loaded in one batch (up to 256
// records in all), so the scan is one memory round trip, not one per record.
template <int NT>
__device__ __forceinline__ Cand scan_records(const Cand *rec, const ulonglong2 *vals, int G,
                                             int stid, unsigned long long *tag) {
    constexpr int R = NT >= 256 ? 1 : 256 / NT;
    Cand e = cand_empty();
    unsigned long long et = 0ull;
    for (int k0 = stid; k0 < G; k0 += R * NT) {
        ulonglong2 rb[R];
        unsigned long long vb[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int k = k0 + u * NT;
            rb[u] = k < G ? __ldcg(reinterpret_cast<const ulonglong2 *>(rec) + k)
                          : make_ulonglong2(~0ull, ~0ull);
            vb[u] = vals != nullptr && k < G ? __ldcg(&vals[k].x) : (unsigned long long)k;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (k0 + u * NT >= G) break;
            const Cand r = unpack_cand(rb[u]);
            if (cand_less(r, e)) {
                e = r;
                et = vb[u];
            }
        }
    }
    *tag = et;
    return e;
}

// Bounded wait of one thread until *ctr reaches target; false when it ran out
// or another CTA reported a timeout.
__device__ __forceinline__ bool wait_ctr(unsigned *ctr, unsigned target, int *err,
                                         long long spin_limit) {
    const long long t0 = clock64();
    while ((int)(ld_acquire(ctr) - target) < 0) {
        if (clock64() - t0 > spin_limit || *(volatile int *)err) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}

// Selection-group minimum of a candidate and its 64-bit payload: the warps'
// minima go through sc[]/sq[] (SW entries) and a named barrier; every
// selection thread gets the result.
template <int SW>
__device__ __forceinline__ Cand sel_min(Cand c, unsigned long long q, Cand *sc,
                                        unsigned long long *sq, unsigned long long *pq) {
    const int lane = threadIdx.x & 31, sw = (threadIdx.x >> 5) % SW;
    Cand r;
    const int src = warp_argmin(c.vk, c.key, &r.vk, &r.key);
    r.idx = __shfl_sync(0xffffffffu, c.idx, src);
    const unsigned long long rq = __shfl_sync(0xffffffffu, q, src);
    if (lane == 0) {
        sc[sw] = r;
        sq[sw] = rq;
    }
    named_sync(2, 32 * SW);
    Cand b = sc[0];
    unsigned long long bq = sq[0];
#pragma unroll
    for (int w = 1; w < SW; ++w)
        if (cand_less(sc[w], b)) {
            b = sc[w];
            bq = sq[w];
        }
    named_sync(2, 32 * SW);  // sc/sq free again
    if (pq) *pq = bq;
    return b;
}

// Selection-group minimum and sum of two 32-bit values (min of a, sum of b).
template <int SW>
__device__ __forceinline__ void sel_min_sum(unsigned a, unsigned b, unsigned *sa, unsigned *sb,
                                            unsigned *ra, unsigned *rb) {
    const int lane = threadIdx.x & 31, sw = (threadIdx.x >> 5) % SW;
    a = __reduce_min_sync(0xffffffffu, a);
    b = __reduce_add_sync(0xffffffffu, b);
    if (lane == 0) {
        sa[sw] = a;
        sb[sw] = b;
    }
    named_sync(2, 32 * SW);
    unsigned ma = sa[0], mb = sb[0];
#pragma unroll
    for (int w = 1; w < SW; ++w) {
        ma = sa[w] < ma ? sa[w] : ma;
        mb += sb[w];
    }
    named_sync(2, 32 * SW);
    *ra = ma;
    *rb = mb;
}

// Selection-group minimum of a 64-bit value.
template <int SW>
__device__ __forceinline__ unsigned long long sel_min_u64(unsigned long long v,
                                                          unsigned long long *sq) {
    const int lane = threadIdx.x & 31, sw = (threadIdx.x >> 5) % SW;
    v = warp_min_u64(v);
    if (lane == 0) sq[sw] = v;
    named_sync(2, 32 * SW);
    unsigned long long r = sq[0];
#pragma unroll
    for (int w = 1; w < SW; ++w) r = sq[w] < r ? sq[w] : r;
    named_sync(2, 32 * SW);
    return r;
}

// SW selection warps; SW == 2 runs the double-buffered mode, SW == 4 in place.
template <typename T, int SW>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pivot_pipe_kernel(LpDesc *__restrict__ d, int W, long long spin_limit, long long budget,
                      int dbm) {
    typedef typename Vec<T>::type V;
    constexpr int VW = Vec<T>::W;
    constexpr int kSelThreads = 32 * SW;  // the last SW warps select
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Cand rbuf[2][32];
    __shared__ unsigned long long ubuf[32];
    __shared__ Cand wpart[32];
    __shared__ Cand selc[SW];
    __shared__ unsigned long long selq[SW];
    __shared__ unsigned sela[SW], selb[SW];
    __shared__ int s_flag, s_p, s_q, s_status, s_jv, s_uok, s_rzero, s_sok, s_abort;

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
    // update threads; the last SW warps select (the launch reserves
    // kSelThreadsMax threads for them, the rest of those update)
    const int NU = B - kSelThreads;
    const int lane = tid & 31;
    const bool selw = tid >= NU;
    const int stid = tid - NU;
    // in place, or double-buffered (dbm; T2 is the second buffer): pivot k
    // reads bufs[cur] and writes bufs[cur ^ 1], with a grid barrier after
    // each pivot
    const bool db = dbm != 0 && d->T2 != nullptr;
    T *bufs[2] = {reinterpret_cast<T *>(d->T), reinterpret_cast<T *>(db ? d->T2 : d->T)};
    int cur = 0;
    const T *Tab = bufs[0];
    const long long P = d->P;
    const int m = d->m, M = d->M, N = d->N;
    int *__restrict__ basis = d->basis;
    const int bland_after = d->bland_after;
    const unsigned long long lim_p = okey((T)d->eps_p);
    const unsigned long long lim_d = okey((T)(-d->eps_d));
    const unsigned long long zero_k = okey((T)0);
    long long iters = d->iters;
    const long long iter_limit =
        iters > 0x3fffffffffffffffll - budget ? 0x3fffffffffffffffll : iters + budget;
    int deg = d->deg;
    int status = ST_RUNNING;
    unsigned *pcnt = d->bar + 64, *rcnt = d->bar + 128;

    // strip and thread map of the update threads
    const int c0 = g * W;  // < P: the host launches ceil(P / W) CTAs
    const int c1 = (int)min((long long)c0 + W, P);
    const int vpr = (c1 - c0) / VW;
    const int rpp = NU / vpr;  // >= 1: the host keeps W <= NU * VW
    const int lr = tid / vpr, lv = tid - lr * vpr;
    const bool active = !selw && lr < rpp;
    const int col0 = c0 + lv * VW;
    // the vector of this strip holding the rhs column, or -1
    const int rv = (N - 1 >= c0 && N - 1 < c1) ? (N - 1 - c0) / VW : -1;
    // scratch: the strip of the pivot row in shared memory; the pivot columns
    // of this and the next pivot, the rhs column of the current tableau (kept
    // here from pivot to pivot, so the selection never reads it from the
    // tableau) and the screening keys in shared memory, or in this CTA's
    // slice of global scratch
    T *sprow = reinterpret_cast<T *>(smem_raw);
    unsigned char *sc = d->scratch_stride > 0
                            ? reinterpret_cast<unsigned char *>(d->scratch) +
                                  (size_t)g * (size_t)d->scratch_stride
                            : smem_raw + (((size_t)W * sizeof(T) + 15) & ~(size_t)15);
    const size_t cbytes = ((size_t)M * sizeof(T) + 15) & ~(size_t)15;
    T *scol[2] = {reinterpret_cast<T *>(sc), reinterpret_cast<T *>(sc + cbytes)};
    T *srhs = reinterpret_cast<T *>(sc + 2 * cbytes);
    unsigned long long *srk = reinterpret_cast<unsigned long long *>(sc + 3 * cbytes);

    // ---- selection of the first pivot from the current tableau (all threads) ----
    int p = -1, q = -1;
    {
        const int bland = deg >= bland_after;
        Cand c = cand_empty();
        const T *z = Tab + (long long)m * P;
        for (int j = c0 + tid; j < c1 && j < N - 1; j += B) {
            const unsigned long long zk = okey(lds(z + j));
            if (zk < lim_d) cand_take(c, bland ? zero_k : zk, j, j);
        }
        c = block_min_c(c, rbuf[0]);
        if (tid == 0) d->part_sel[g] = c;
        if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) status = ST_TIMEOUT;
        if (status == ST_RUNNING) {
            const Cand sel = load_partials_min(d->part_sel, G, rbuf[1]);
            if (sel.idx < 0) status = ST_OPTIMAL;
            else if (iters >= iter_limit) status = ST_ITER_LIMIT;
            else if (sel.idx >= N - 1) status = ST_TIMEOUT;  // never: a partial from outside the row
            else q = sel.idx;
        }
        if (status == ST_RUNNING) {
            // the whole pivot column and the ratio test, in every CTA
            unsigned long long lmin = ~0ull;
            for (int i = tid; i < M; i += B) {
                const T a = lds(Tab + (long long)i * P + q);
                scol[0][i] = a;
                if (i < m) {
                    const T rhs = lds(Tab + (long long)i * P + (N - 1));
                    const unsigned long long rk =
                        okey(a) > lim_p ? screen_key(pos_part(rhs), a) : ~0ull;
                    srhs[i] = rhs;
                    srk[i] = rk;
                    lmin = rk < lmin ? rk : lmin;
                }
            }
            const unsigned long long rstar = block_min_u(lmin, ubuf);
            if (rstar == ~0ull) {
                status = ST_UNBOUNDED;
            } else {
                const unsigned long long thr = screen_thr(rstar, (T)0);
                Cand rc = cand_empty();
                for (int i = tid; i < m; i += B)
                    if (srk[i] <= thr)
                        cand_take(rc, okey(pos_part(srhs[i]) / scol[0][i]), bland ? __ldcg(basis + i) : i, i);
                rc = block_min_c(rc, rbuf[0]);
                p = rc.idx;
                deg = (rc.vk == zero_k) ? deg + 1 : 0;
            }
        }
    }

    int lk = 0;  // pivots made in this launch (parity of records and pivot-column buffers)
    const int rowner = (N - 1) / W;  // the CTA whose strip holds the rhs column
    while (status == ST_RUNNING) {
        const int ab = tid == 0 ? abort_peek(d->abort) : 0;  // used at the pass's end
        const T *A = bufs[cur];
        T *Bn = bufs[cur ^ 1];
        const T *col = scol[lk & 1];
        T *ncol = scol[(lk + 1) & 1];
        const int par = (lk + 1) & 1;  // records of the selection of pivot k+1
        Cand *psel = d->part_sel + par * G;
        ulonglong2 *pval = reinterpret_cast<ulonglong2 *>(d->part_vals) + par * G;
        const unsigned target = (unsigned)G * (unsigned)(lk + 1);
        const int nbland = deg >= bland_after;  // rule of pivot k+1's selection
        if (!selw) {
            const T piv = col[p];
            // the strip of the objective row is loaded with the pivot row's:
            // both head the chain to the next pricing record
            V zt;
            const bool zown = tid < vpr;
            if (zown) zt = ldv(reinterpret_cast<const V *>(A + (long long)m * P + c0 + tid * VW));
            // Step 4 on this CTA's strip of the pivot row
            for (int j = c0 + tid; j < c1; j += NU)
                sprow[j - c0] = lds(A + (long long)p * P + j) / piv;
            named_sync(1, NU);
            // the new strip of the objective row, held back in registers, and
            // the CTA's pricing candidate for pivot k+1
            Cand c = cand_empty();
            if (zown) {
                const T colm = col[m];
                const V pr = *reinterpret_cast<const V *>(sprow + tid * VW);
                vfma(zt, colm, pr);
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    const int j = c0 + tid * VW + k;
                    const unsigned long long zk = okey(getc(zt, k));
                    if (j < N - 1 && zk < lim_d) cand_take(c, nbland ? zero_k : zk, j, j);
                }
            }
            c = warp_min(c);
            if (lane == 0) wpart[tid >> 5] = c;
            named_sync(1, NU);
            if (tid < 32) {  // warp 0 reduces the warps' candidates and publishes
                const Cand e = tid < NU / 32 ? wpart[tid] : cand_empty();
                const Cand r = warp_min(e);
                if (tid == 0) {
                    psel[g] = r;
                    // with it, the new pivot-row values the selection needs
                    // from this strip: at the candidate column and at the rhs
                    pval[g] = make_ulonglong2(r.idx >= 0 ? tbits(sprow[r.idx - c0]) : 0ull,
                                              rv >= 0 ? tbits(sprow[N - 1 - c0]) : 0ull);
                    red_add_release(pcnt, 1u);
                    s_jv = (r.idx >= 0 && !db) ? (r.idx - c0) / VW : -1;
                }
            }
            named_sync(1, NU);
            const int jv = s_jv;  // protected: the vector of the CTA's candidate
            if (zown && tid != jv)
                *reinterpret_cast<V *>(Bn + (long long)m * P + c0 + tid * VW) = zt;
            // Step 5 on the constraint rows of the strip, but the protected vectors
            if (active && lv != jv) {
                const V pr = *reinterpret_cast<const V *>(sprow + lv * VW);
                const T *abase = A + col0;
                T *bbase = Bn + col0;
                int i = lr;
                for (; i + 3 * rpp < m; i += 4 * rpp) {
                    const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                    const V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    const V t1 = ldv(reinterpret_cast<const V *>(abase + (long long)i1 * P));
                    const V t2 = ldv(reinterpret_cast<const V *>(abase + (long long)i2 * P));
                    const V t3 = ldv(reinterpret_cast<const V *>(abase + (long long)i3 * P));
                    const T a0 = col[i], a1 = col[i1], a2 = col[i2], a3 = col[i3];
                    *reinterpret_cast<V *>(bbase + (long long)i * P) = pivot_vec<T>(t0, i, p, a0, pr);
                    *reinterpret_cast<V *>(bbase + (long long)i1 * P) = pivot_vec<T>(t1, i1, p, a1, pr);
                    *reinterpret_cast<V *>(bbase + (long long)i2 * P) = pivot_vec<T>(t2, i2, p, a2, pr);
                    *reinterpret_cast<V *>(bbase + (long long)i3 * P) = pivot_vec<T>(t3, i3, p, a3, pr);
                }
                for (; i < m; i += rpp) {
                    const V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    *reinterpret_cast<V *>(bbase + (long long)i * P) =
                        pivot_vec<T>(t0, i, p, col[i], pr);
                }
            }
            // in place: every CTA's selection is done reading the protected
            // vector, then update it (double-buffered: nothing to protect)
            if (tid == 0) s_uok = db ? 1 : (int)wait_ctr(rcnt, target, d->err, spin_limit);
            named_sync(1, NU);
            if (s_uok && !db && jv >= 0) {
                const V vpr_ = *reinterpret_cast<const V *>(sprow + jv * VW);
                T *vbase = Bn + c0 + jv * VW;
                for (int i = tid; i < M; i += NU) {
                    V *p0 = reinterpret_cast<V *>(vbase + (long long)i * P);
                    *p0 = pivot_vec<T>(ldv(p0), i, p, col[i], vpr_);
                }
            }
        } else {
            // selection of pivot k+1, overlapping the update of pivot k
            int st = ST_RUNNING, np = -1, nq = -1, rzero = 0;
            if (stid == 0) {
                int ok = 1;
                if (g == 0) {
                    // the basis and trace of pivot k, once every CTA's selection
                    // of pivot k is done reading the basis of pivot k-1
                    ok = (int)wait_ctr(rcnt, target - (unsigned)G, d->err, spin_limit);
                    if (ok) {
                        if (iters < d->trace_cap) {
                            d->trace[2 * iters] = p;
                            d->trace[2 * iters + 1] = q;
                        }
                        basis[p] = q;
                        d->last_p = p;
                        d->last_q = q;
                    }
                }
                // every CTA has finished pivot k-1 and published its record
                if (ok) ok = (int)wait_ctr(pcnt, target, d->err, spin_limit);
                s_sok = ok;
            }
            named_sync(2, kSelThreads);
            if (!s_sok) {
                st = ST_TIMEOUT;
            } else {
                // Step 2: the entering column from the G pricing records
                unsigned long long eq;
                const Cand e = scan_records<kSelThreads>(psel, pval, G, stid, &eq);
                const unsigned long long prr_b = __ldcg(&pval[rowner].y);
                unsigned long long prq_b;
                const Cand sel = sel_min<SW>(e, eq, selc, selq, &prq_b);
                if (sel.idx < 0) st = ST_OPTIMAL;
                else if (iters + 1 >= iter_limit) st = ST_ITER_LIMIT;
                else if (sel.idx >= N - 1) st = ST_TIMEOUT;  // never: a record from outside the row
                else nq = sel.idx;
                if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                if (st == ST_RUNNING) {
                    // column q' and rhs of tableau k+1, every row, and Step 3
                    const T prq = tfrom<T>(prq_b), prr = tfrom<T>(prr_b);
                    unsigned long long lmin = ~0ull;
                    // kColRows constraint rows per thread in flight (the loads
                    // are L2 round trips); the objective row's entry rides
                    // with the first batch, so that m = 2^k rows take 2^k /
                    // (kColRows * kSelThreads) batches, not one more
                    const T am = stid == 0 ? lds(A + (long long)m * P + nq) : (T)0;
                    for (int i0 = stid; i0 < m; i0 += kColRows * kSelThreads) {
                        T av[kColRows];
#pragma unroll
                        for (int u = 0; u < kColRows; ++u) {
                            const int i = i0 + u * kSelThreads;
                            av[u] = i < m ? lds(A + (long long)i * P + nq) : (T)0;
                        }
#pragma unroll
                        for (int u = 0; u < kColRows; ++u) {
                            const int i = i0 + u * kSelThreads;
                            if (i >= m) break;
                            const T ci = col[i];
                            const T a = (i == p) ? prq : tfma(-ci, prq, av[u]);
                            ncol[i] = a;
                            const T rhs = (i == p) ? prr : tfma(-ci, prr, srhs[i]);
                            srhs[i] = rhs;
                            const unsigned long long rk =
                                okey(a) > lim_p ? screen_key(pos_part(rhs), a) : ~0ull;
                            srk[i] = rk;
                            lmin = rk < lmin ? rk : lmin;
                        }
                    }
                    if (stid == 0) ncol[m] = tfma(-col[m], prq, am);  // p < m
                    const unsigned long long rstar = sel_min_u64<SW>(lmin, selq);
                    if (rstar == ~0ull) {
                        st = ST_UNBOUNDED;
                    } else {
                        // the rows within the screening threshold: when there is
                        // one it is the exact minimum, otherwise compare their
                        // exact quotients, then keys
                        const unsigned long long thr = screen_thr(rstar, (T)0);
                        unsigned first = 0xffffffffu, cnt = 0;
                        for (int i = stid; i < m; i += kSelThreads)
                            if (srk[i] <= thr) {
                                first = (unsigned)i < first ? (unsigned)i : first;
                                ++cnt;
                            }
                        unsigned gfirst, gcnt;
                        sel_min_sum<SW>(first, cnt, sela, selb, &gfirst, &gcnt);
                        if (gcnt == 1) {
                            np = (int)gfirst;
                            rzero = srk[np] == zero_k;  // screening keys are exact at +0
                        } else {
                            Cand rc = cand_empty();
                            for (int i = stid; i < m; i += kSelThreads)
                                if (srk[i] <= thr) {
                                    const T nm = pos_part(srhs[i]);
                                    const unsigned long long vk =
                                        tbits(nm) == 0ull ? zero_k : okey(nm / ncol[i]);
                                    const int key = nbland ? (i == p ? q : __ldcg(basis + i)) : i;
                                    cand_take(rc, vk, key, i);
                                }
                            rc = sel_min<SW>(rc, 0ull, selc, selq, nullptr);
                            np = rc.idx;
                            rzero = rc.vk == zero_k;
                        }
                    }
                }
            }
            // every selection thread of this CTA is done reading tableau k: arrive
            // (also when no ratio test ran: the owners of protected vectors wait)
            named_sync(2, kSelThreads);
            if (stid == 0) {
                if (st != ST_TIMEOUT) red_add_release(rcnt, 1u);
                s_status = st;
                s_p = np;
                s_q = nq;
                s_rzero = rzero;
            }
        }
        // the CTA's update of pivot k and its selection of pivot k+1 are done
        if (tid == 0) {
            s_abort = ab;  // past the host's deadline: stop, and end every CTA's waits
            if (ab) atomicExch(d->err, 1);
        }
        __syncthreads();
        ++iters;
        ++lk;
        status = s_abort ? ST_TIMEOUT : s_status;
        if (!s_uok) status = ST_TIMEOUT;
        if (status == ST_RUNNING) {
            p = s_p;
            q = s_q;
            deg = s_rzero ? deg + 1 : 0;
        }
        if (db) {
            cur ^= 1;
            // keeps the CTAs in step: their row streams then share DRAM pages
            if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) {
                status = ST_TIMEOUT;
                break;
            }
        }
    }

    if (g == 0 && tid == 0) {
        d->status = (*(volatile int *)d->err) ? ST_TIMEOUT : status;
        d->iters = iters;
        d->iter_limit = iter_limit;
        d->deg = deg;
        if (db) {  // hand over the buffer holding the last tableau as the current one
            d->T = bufs[cur];
            d->T2 = bufs[cur ^ 1];
        }
    }
}

// ---------------------------------------------------------------------------
// Pipelined dual simplex for the dual form (sense LP_MIN_GE), double-buffered:
// pivot k reads bufs[cur] and writes bufs[cur ^ 1], so the selection of pivot
// k+1 reads tableau k while the update warps stream pivot k.
//   update warps     divide the strip of the pivot row (Step 4), update the
//                    strip of the objective row (kept for the selection) and
//                    the rest of the strip (Step 5);
//   selection warps  form the rhs of tableau k+1 over every row and take the
//                    leaving row r' (the most negative rhs; every CTA does this
//                    redundantly), then row r' of tableau k+1 on the CTA's own
//                    strip and the dual ratio test on it, publish the strip's
//                    winner with its pivot-row value, reduce the G records to
//                    the entering column q', and form column q' of tableau k+1
//                    (the next pivot column) in the CTA's scratch.
// The values the selection forms are the very fma results the update writes.
// A grid barrier ends each pivot.  The first pivot's selection runs alone.
template <typename T, int SW>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pivot_pipe_dual_kernel(LpDesc *__restrict__ d, int W, long long spin_limit, long long budget) {
    typedef typename Vec<T>::type V;
    constexpr int VW = Vec<T>::W;
    constexpr int kSelThreads = 32 * SW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Cand rbuf[2][32];
    __shared__ Cand selc[SW];
    __shared__ unsigned long long selq[SW];
    __shared__ int s_flag, s_p, s_q, s_status, s_rzero, s_sok, s_abort;

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
    const int NU = B - kSelThreads;  // update threads; the last SW warps select
    const bool selw = tid >= NU;
    const int stid = tid - NU;
    T *bufs[2] = {reinterpret_cast<T *>(d->T), reinterpret_cast<T *>(d->T2)};
    int cur = 0;
    const long long P = d->P;
    const int m = d->m, M = d->M, N = d->N;
    int *__restrict__ basis = d->basis;
    const int bland_after = d->bland_after;
    const unsigned long long lim_np = okey((T)(-d->eps_p));
    const unsigned long long lim_r = okey((T)(-d->eps_r));
    const unsigned long long zero_k = okey((T)0);
    long long iters = d->iters;
    const long long iter_limit =
        iters > 0x3fffffffffffffffll - budget ? 0x3fffffffffffffffll : iters + budget;
    int deg = d->deg;
    int status = ST_RUNNING;
    unsigned *rcnt = d->bar + 128;

    // strip and thread map of the update threads
    const int c0 = g * W;  // < P: the host launches ceil(P / W) CTAs
    const int c1 = (int)min((long long)c0 + W, P);
    const int jend = min(c1, N - 1);  // the strip's columns that may enter
    const int vpr = (c1 - c0) / VW;
    const int rpp = NU / vpr;  // >= 1: the host keeps W <= NU * VW
    const int lr = tid / vpr, lv = tid - lr * vpr;
    const bool active = !selw && lr < rpp;
    const int col0 = c0 + lv * VW;
    // scratch: the strip of the pivot row in shared memory; the strip of the
    // new objective row and the pivot columns of this and the next pivot in
    // shared memory, or in this CTA's slice of global scratch
    T *sprow = reinterpret_cast<T *>(smem_raw);
    const size_t wbytes = ((size_t)W * sizeof(T) + 15) & ~(size_t)15;
    unsigned char *sc = d->scratch_stride > 0
                            ? reinterpret_cast<unsigned char *>(d->scratch) +
                                  (size_t)g * (size_t)d->scratch_stride
                            : smem_raw + wbytes;
    const size_t cbytes = ((size_t)M * sizeof(T) + 15) & ~(size_t)15;
    T *sz = reinterpret_cast<T *>(sc);
    T *scol[2] = {reinterpret_cast<T *>(sc + wbytes), reinterpret_cast<T *>(sc + wbytes + cbytes)};

    // ---- selection of the first pivot from the current tableau (all threads) ----
    int p = -1, q = -1;
    {
        const T *A = bufs[0];
        const int bland = deg >= bland_after;
        // leaving row, in every CTA over all rows
        Cand c = cand_empty();
        for (int i = tid; i < m; i += B) {
            const unsigned long long vk = okey(lds(A + (long long)i * P + (N - 1)));
            if (vk < lim_r) cand_take(c, bland ? zero_k : vk, bland ? __ldcg(basis + i) : i, i);
        }
        c = block_min_c(c, rbuf[0]);
        if (c.idx < 0) status = ST_OPTIMAL;
        else if (iters >= iter_limit) status = ST_ITER_LIMIT;
        else p = c.idx;
        if (status == ST_RUNNING) {
            // entering column: the dual ratio test on this CTA's strip of row
            // p, then over the CTAs' partials
            const T *rowr = A + (long long)p * P, *z = A + (long long)m * P;
            Cand e = cand_empty();
            for (int j = c0 + tid; j < jend; j += B) {
                const T a = lds(rowr + j);
                if (okey(a) < lim_np) cand_take(e, okey(pos_part(lds(z + j)) / neg(a)), j, j);
            }
            e = block_min_c(e, rbuf[1]);
            if (tid == 0) d->part_sel[g] = e;
            if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) status = ST_TIMEOUT;
            if (status == ST_RUNNING) {
                const Cand sel = load_partials_min(d->part_sel, G, rbuf[0]);
                if (sel.idx < 0) {
                    status = ST_INFEASIBLE;
                } else if (sel.idx >= N - 1) {
                    status = ST_TIMEOUT;  // never: a partial from outside the row
                } else {
                    q = sel.idx;
                    deg = (sel.vk == zero_k) ? deg + 1 : 0;
                    for (int i = tid; i < M; i += B) scol[0][i] = lds(A + (long long)i * P + q);
                }
            }
        }
    }
    __syncthreads();  // the first pivot column is in scol[0]

    int lk = 0;  // pivots made in this launch (parity of records and pivot columns)
    while (status == ST_RUNNING) {
        const int ab = tid == 0 ? abort_peek(d->abort) : 0;  // used at the pass's end
        const T *A = bufs[cur];
        T *Bn = bufs[cur ^ 1];
        const T *col = scol[lk & 1];
        T *ncol = scol[(lk + 1) & 1];
        const int par = (lk + 1) & 1;  // records of the selection of pivot k+1
        Cand *psel = d->part_sel + par * G;
        ulonglong2 *pval = reinterpret_cast<ulonglong2 *>(d->part_vals) + par * G;
        const unsigned target = (unsigned)G * (unsigned)(lk + 1);
        if (g == 0 && tid == 0) {  // grid barriers order this against every reader
            if (iters < d->trace_cap) {
                d->trace[2 * iters] = p;
                d->trace[2 * iters + 1] = q;
            }
            basis[p] = q;
            d->last_p = p;
            d->last_q = q;
        }
        const int nbland = deg >= bland_after;  // rule of pivot k+1's selection
        const T piv = col[p];
        if (!selw) {
            // the strip of the objective row is loaded with the pivot row's
            V zt;
            if (tid < vpr) zt = ldv(reinterpret_cast<const V *>(A + (long long)m * P + c0 + tid * VW));
            // Step 4 on this CTA's strip of the pivot row
            for (int j = c0 + tid; j < c1; j += NU)
                sprow[j - c0] = lds(A + (long long)p * P + j) / piv;
            named_sync(1, NU);
            // the new strip of the objective row, also kept for the selection
            if (tid < vpr) {
                const T colm = col[m];
                const V pr = *reinterpret_cast<const V *>(sprow + tid * VW);
                vfma(zt, colm, pr);
                *reinterpret_cast<V *>(Bn + (long long)m * P + c0 + tid * VW) = zt;
                *reinterpret_cast<V *>(sz + tid * VW) = zt;
            }
            named_sync(3, B);  // sprow and sz ready for the selection warps
            // Step 5 on the constraint rows of the strip
            if (active) {
                const V pr = *reinterpret_cast<const V *>(sprow + lv * VW);
                const T *abase = A + col0;
                T *bbase = Bn + col0;
                int i = lr;
                for (; i + 3 * rpp < m; i += 4 * rpp) {
                    const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                    const V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    const V t1 = ldv(reinterpret_cast<const V *>(abase + (long long)i1 * P));
                    const V t2 = ldv(reinterpret_cast<const V *>(abase + (long long)i2 * P));
                    const V t3 = ldv(reinterpret_cast<const V *>(abase + (long long)i3 * P));
                    const T a0 = col[i], a1 = col[i1], a2 = col[i2], a3 = col[i3];
                    *reinterpret_cast<V *>(bbase + (long long)i * P) = pivot_vec<T>(t0, i, p, a0, pr);
                    *reinterpret_cast<V *>(bbase + (long long)i1 * P) = pivot_vec<T>(t1, i1, p, a1, pr);
                    *reinterpret_cast<V *>(bbase + (long long)i2 * P) = pivot_vec<T>(t2, i2, p, a2, pr);
                    *reinterpret_cast<V *>(bbase + (long long)i3 * P) = pivot_vec<T>(t3, i3, p, a3, pr);
                }
                for (; i < m; i += rpp) {
                    const V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    *reinterpret_cast<V *>(bbase + (long long)i * P) =
                        pivot_vec<T>(t0, i, p, col[i], pr);
                }
            }
        } else {
            // selection of pivot k+1, overlapping the update of pivot k
            int st = ST_RUNNING, np = -1, nq = -1, rzero = 0;
            // leaving row: the rhs of tableau k+1 over every row
            const T prr = lds(A + (long long)p * P + (N - 1)) / piv;
            Cand c = cand_empty();
            for (int i0 = stid; i0 < m; i0 += kSelRows * kSelThreads) {
                T hv[kSelRows];
#pragma unroll
                for (int u = 0; u < kSelRows; ++u) {
                    const int i = i0 + u * kSelThreads;
                    hv[u] = i < m ? lds(A + (long long)i * P + (N - 1)) : (T)0;
                }
#pragma unroll
                for (int u = 0; u < kSelRows; ++u) {
                    const int i = i0 + u * kSelThreads;
                    if (i >= m) break;
                    const T rhs = (i == p) ? prr : tfma(-col[i], prr, hv[u]);
                    const unsigned long long vk = okey(rhs);
                    if (vk < lim_r)
                        cand_take(c, nbland ? zero_k : vk,
                                  nbland ? (i == p ? q : __ldcg(basis + i)) : i, i);
                }
            }
            c = sel_min<SW>(c, 0ull, selc, selq, nullptr);
            if (c.idx < 0) st = ST_OPTIMAL;
            else if (iters + 1 >= iter_limit) st = ST_ITER_LIMIT;
            else if (c.idx >= m) st = ST_TIMEOUT;  // never: a row outside the tableau
            else np = c.idx;
            if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
            named_sync(3, B);  // the update warps' sprow and sz
            if (st == ST_RUNNING) {
                // row r' of tableau k+1 on this strip and the dual ratio test
                const T cr = col[np];
                Cand e = cand_empty();
                unsigned long long eq = 0ull;
                for (int j = c0 + stid; j < jend; j += kSelThreads) {
                    const T pr = sprow[j - c0];
                    const T a = (np == p) ? pr : tfma(-cr, pr, lds(A + (long long)np * P + j));
                    if (okey(a) < lim_np) {
                        const unsigned long long vk = okey(pos_part(sz[j - c0]) / neg(a));
                        if (vk < e.vk || (vk == e.vk && j < e.key)) {
                            e.vk = vk;
                            e.key = j;
                            e.idx = j;
                            eq = tbits(pr);
                        }
                    }
                }
                e = sel_min<SW>(e, eq, selc, selq, &eq);
                if (stid == 0) {
                    psel[g] = e;
                    pval[g] = make_ulonglong2(eq, 0ull);
                }
            }
            named_sync(2, kSelThreads);
            if (stid == 0 && st != ST_TIMEOUT) red_add_release(rcnt, 1u);
            if (st == ST_RUNNING) {
                if (stid == 0) s_sok = (int)wait_ctr(rcnt, target, d->err, spin_limit);
                named_sync(2, kSelThreads);
                if (!s_sok) {
                    st = ST_TIMEOUT;
                } else {
                    // entering column from the G records, with its pivot-row value
                    unsigned long long eq;
                    const Cand e = scan_records<kSelThreads>(psel, pval, G, stid, &eq);
                    unsigned long long prq_b;
                    const Cand sel = sel_min<SW>(e, eq, selc, selq, &prq_b);
                    if (sel.idx < 0) {
                        st = ST_INFEASIBLE;
                    } else if (sel.idx >= N - 1) {  // never: a record from outside the row
                        if (stid == 0) atomicExch(d->err, 1);
                        st = ST_TIMEOUT;
                    } else {
                        nq = sel.idx;
                        rzero = sel.vk == zero_k;
                        // column q' of tableau k+1: the next pivot column
                        const T prq = tfrom<T>(prq_b);
                        // the objective row's entry rides with the first batch
                        const T am = stid == 0 ? lds(A + (long long)m * P + nq) : (T)0;
                        for (int i0 = stid; i0 < m; i0 += kSelRows * kSelThreads) {
                            T av[kSelRows];
#pragma unroll
                            for (int u = 0; u < kSelRows; ++u) {
                                const int i = i0 + u * kSelThreads;
                                av[u] = i < m ? lds(A + (long long)i * P + nq) : (T)0;
                            }
#pragma unroll
                            for (int u = 0; u < kSelRows; ++u) {
                                const int i = i0 + u * kSelThreads;
                                if (i >= m) break;
                                ncol[i] = (i == p) ? prq : tfma(-col[i], prq, av[u]);
                            }
                        }
                        if (stid == 0) ncol[m] = tfma(-col[m], prq, am);  // p < m
                    }
                }
            }
            if (stid == 0) {
                s_status = st;
                s_p = np;
                s_q = nq;
                s_rzero = rzero;
            }
        }
        // the CTA's update of pivot k and its selection of pivot k+1 are done
        if (tid == 0) {
            s_abort = ab;  // past the host's deadline: stop, and end every CTA's waits
            if (ab) atomicExch(d->err, 1);
        }
        __syncthreads();
        ++iters;
        ++lk;
        status = s_abort ? ST_TIMEOUT : s_status;
        if (status == ST_RUNNING) {
            p = s_p;
            q = s_q;
            deg = s_rzero ? deg + 1 : 0;
        }
        cur ^= 1;
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
        d->T = bufs[cur];  // hand over the buffer holding the last tableau
        d->T2 = bufs[cur ^ 1];
    }
}

// ---------------------------------------------------------------------------
// Two pivots per pass (multi-pivot blocking), primal, double-buffered.
//
// A pass reads tableau T0 from bufs[cur] once and writes T2 into bufs[cur^1],
// applying the pass's pivots (p1, q1) and (p2, q2) to every element in the
// order the one-pivot method applies them:
//   t = i == p1 ? prow1[j] : fma(-col1[i], prow1[j], T0[i][j]);
//   T2[i][j] = i == p2 ? prow2[j] : fma(-col2[i], prow2[j], t),
// so the result is bit for bit that of two one-pivot passes, with half of
// their tableau traffic.  prow1 = T0[p1][.] / col1[p1] and prow2 = T1[p2][.] /
// col2[p2] are formed per strip at the start of the pass; col1 and col2 (the
// columns q1 of T0 and q2 of T1) come from the previous pass's selection.
//
// While the update warps stream the pass, the selection warps select the
// next two pivots from T0 and the pass's pivots (Steps 2-3 twice):
//   a: pricing records (each CTA's best column of the objective row of T2,
//      with the pass's pivot-row values there and at the rhs) -> q_a; the
//      column q_a and rhs of T2 -> ratio test -> p_a;
//   b: row p_a of T2 on each CTA's strip divided by the pivot (the pivot row
//      of pivot a) and the objective row after pivot a -> pricing records ->
//      q_b; column q_b and rhs after pivot a -> p_b.
// The columns and the ratio test are either formed whole in every CTA, or
// (DIST, tall tableaus) on each CTA's slice of rows with one ratio record per
// CTA (ratio_slices), the whole columns then copied from global slots.
// A pass holds one pivot when the next pivot ends the solve (optimal,
// unbounded, iteration limit); the first pass of a launch holds the first
// pivot alone.
//
// No grid barrier separates the passes: a CTA starts pass k+1 when its own
// pass k is done.  Its pass-k+1 pricing record proves to every reader that
// its strip of T2 is written; before it writes into bufs[cur] again (pass k+1
// writes what pass k read), it waits until every CTA's selection of pass k
// has counted itself done.  That wait overlaps its own start of pass k+1
// (pivot rows, objective row, record), so pass k+1's selection starts
// without waiting for the slowest CTA of pass k.

constexpr int kBlk = 2;       // pivots per pass
constexpr int kBlkVals = 8;   // values per record: [0, 3) at the record's column, [4, 7) at the rhs
                              // (two-pivot primal kernel: [3] the buffer of the column's rows)
constexpr int kRecTab = 4;    // values of a record the selection keeps in shared memory
constexpr int kMaxRecs = 256; // CTAs of a two-pivot launch (records copied to shared memory)

// ---- the columns of one CTA of the two-pivot primal kernel ----
//
// Run A [a0, a0 + wa) and run B [b0, b0 + wb); local column l in [0, wa + wb),
// A first.  Without a split (split == 0) CTA g owns the contiguous strip
// [g W, g W + W), cut at P.  With a split column (a multiple of the sector,
// where the structural columns end), [0, split) and [split, P) are each cut
// into G near-equal runs of whole sectors, one of each per CTA.  The slack
// column of a row whose slack is still basic holds a unit vector: zero in
// every pivot row but its own, so the update leaves it in place (see the
// kernel); split runs give every CTA the same share of the columns that are
// updated.
struct Strip {
    int a0, wa, b0, wb;
    __host__ __device__ int w() const { return wa + wb; }
    __host__ __device__ int lcol(int j) const {
        if ((unsigned)(j - a0) < (unsigned)wa) return j - a0;
        if ((unsigned)(j - b0) < (unsigned)wb) return wa + (j - b0);
        return -1;
    }
};
__host__ __device__ inline Strip make_strip(int g, int G, int W, int split, long long P, int sector) {
    Strip s;
    if (split <= 0) {
        const long long a0 = (long long)g * W;
        s.a0 = (int)a0;
        s.wa = (int)(a0 >= P ? 0 : (a0 + W <= P ? W : P - a0));
        s.b0 = 0;
        s.wb = 0;
        return s;
    }
    const long long nb = P - split;
    const long long ea0 = (long long)split * g / G / sector * sector;
    const long long ea1 = (long long)split * (g + 1) / G / sector * sector;
    const long long eb0 = nb * g / G / sector * sector, eb1 = nb * (g + 1) / G / sector * sector;
    s.a0 = (int)ea0;
    s.wa = (int)(ea1 - ea0);
    s.b0 = (int)(split + eb0);
    s.wb = (int)(eb1 - eb0);
    return s;
}

// OR of a flag over the nthreads threads of named barrier id (which it is).
__device__ __forceinline__ int named_bar_or(int id, int nthreads, int v) {
    unsigned r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\n"
        "bar.red.or.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)v), "r"(id), "r"(nthreads)
        : "memory");
    return (int)r;
}
__device__ __forceinline__ bool not_finite(double x) {
    return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool not_finite(float x) {
    return (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u;
}
// a component of v is -0
__device__ __forceinline__ bool has_negzero(const double2 &v) {
    return (unsigned long long)__double_as_longlong(v.x) == kSign ||
           (unsigned long long)__double_as_longlong(v.y) == kSign;
}
__device__ __forceinline__ bool has_negzero(const float4 &v) {
    return __float_as_uint(v.x) == 0x80000000u || __float_as_uint(v.y) == 0x80000000u ||
           __float_as_uint(v.z) == 0x80000000u || __float_as_uint(v.w) == 0x80000000u;
}
__device__ __forceinline__ bool zero_vec(const double2 &v) {
    return (((unsigned long long)__double_as_longlong(v.x) |
             (unsigned long long)__double_as_longlong(v.y)) << 1) == 0ull;
}
__device__ __forceinline__ bool zero_vec(const float4 &v) {
    return ((__float_as_uint(v.x) | __float_as_uint(v.y) | __float_as_uint(v.z) |
             __float_as_uint(v.w)) << 1) == 0u;
}

// scan_records over one round of two-pivot records, which also copies the
// first NV values of every record (vals + k * kBlkVals) to tab[k * NV + v] in
// shared memory, loaded in the same batch as the records: after the selection
// group's next barrier every thread reads the winner's values from there,
// without another round trip to memory (a round trip costs several
// microseconds while the update streams the tableau).
template <int NT, int NV>
__device__ __forceinline__ Cand scan_records_tab(const Cand *rec, const unsigned long long *vals,
                                                 int G, int stid, unsigned long long *tag,
                                                 unsigned long long *tab) {
    constexpr int R = NT >= 256 ? 1 : 256 / NT;
    Cand e = cand_empty();
    unsigned long long et = 0ull;
    for (int k0 = stid; k0 < G; k0 += R * NT) {
        ulonglong2 rb[R];
        unsigned long long vb[R][NV];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int k = k0 + u * NT;
            rb[u] = k < G ? __ldcg(reinterpret_cast<const ulonglong2 *>(rec) + k)
                          : make_ulonglong2(~0ull, ~0ull);
#pragma unroll
            for (int v = 0; v < NV; ++v) vb[u][v] = k < G ? __ldcg(vals + (size_t)k * kBlkVals + v) : 0ull;
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            const int k = k0 + u * NT;
            if (k >= G) break;
#pragma unroll
            for (int v = 0; v < NV; ++v) tab[k * NV + v] = vb[u][v];
            const Cand r = unpack_cand(rb[u]);
            if (cand_less(r, e)) {
                e = r;
                et = (unsigned long long)k;
            }
        }
    }
    *tag = et;
    return e;
}

// Copy a whole pivot column (cbytes, a multiple of 16, from its global slot)
// into this CTA's scratch: into shared memory asynchronously (cp.async, 16
// bytes per copy; fill_wait completes this thread's copies), into a global
// scratch slice with plain loads.  Rows the CTA formed itself get the bits
// they already hold.
template <typename T>
__device__ __forceinline__ void fill_column(T *dst, const T *src, size_t cbytes, int stid, int nt,
                                            bool smem) {
    const int n16 = (int)(cbytes / 16);
    if (smem) {
        const unsigned base = (unsigned)__cvta_generic_to_shared(dst);
        const char *gsrc = reinterpret_cast<const char *>(src);
        for (int c = stid; c < n16; c += nt)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + 16u * (unsigned)c),
                         "l"(gsrc + 16 * (size_t)c)
                         : "memory");
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    } else {
        const ulonglong2 *s2 = reinterpret_cast<const ulonglong2 *>(src);
        ulonglong2 *d2 = reinterpret_cast<ulonglong2 *>(dst);
        for (int c = stid; c < n16; c += nt) d2[c] = __ldcg(s2 + c);
    }
}
__device__ __forceinline__ void fill_wait() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// ---- the distributed ratio test of the two-pivot primal kernel ----
//
// Every CTA forms the new pivot column, the rhs and the screening keys only on
// its own slice of rows [r0, r1) (rows g*rs .. g*rs + rs - 1), writes its part
// of the column to a global slot, and publishes one ratio record per round:
// {smallest key of the slice, (count << 32 | first row) of its rows within the
// screening threshold of that key, the column's entry at that row}.  From all
// records every CTA takes the same decision: with rstar the smallest key and
// thr its threshold, the slices whose key is within thr hold every row within
// thr, each at least one, and a slice's count covers its rows within thr
// (its own threshold is at least thr); so the sum of their counts is 1
// exactly when one row in all is within thr, which is then the leaving row,
// as in the one-CTA test.  Otherwise (near ties) the slices' exact quotients
// go through a second exchange.  Either way the row and its keys are those of
// the screened test over all rows.
struct RatioPick {
    int status;               // ST_RUNNING, ST_UNBOUNDED or ST_TIMEOUT
    int row;                  // the leaving row, or -1: near ties, exact round needed
    unsigned long long key;   // the smallest screening key (rstar)
    unsigned long long val;   // bits of the new column's entry at row
};

template <typename T, int SW>
__device__ RatioPick ratio_slices(unsigned long long lmin, const unsigned long long *srk,
                                  const T *ncol, int r0, int r1, int rs, unsigned long long *recs,
                                  unsigned *cnt, unsigned target, int *err, long long spin_limit,
                                  int G, int g, int stid, unsigned long long *selq, unsigned *sela,
                                  unsigned *selb, unsigned long long *vtab, volatile int *s_ok) {
    constexpr int NT = 32 * SW;
    constexpr int R = NT >= 256 ? 1 : 256 / NT;  // G <= 256
    RatioPick out{ST_RUNNING, -1, ~0ull, 0ull};
    // this slice's record
    const unsigned long long kmin = sel_min_u64<SW>(lmin, selq);
    unsigned first = 0xffffffffu, cnt_g = 0;
    if (kmin != ~0ull) {
        const unsigned long long thr = screen_thr(kmin, (T)0);
        for (int i = r0 + stid; i < r1; i += NT)
            if (srk[i] <= thr) {
                first = (unsigned)i < first ? (unsigned)i : first;
                ++cnt_g;
            }
    }
    unsigned sfirst, scnt;
    sel_min_sum<SW>(first, cnt_g, sela, selb, &sfirst, &scnt);
    if (stid == 0) {
        unsigned long long *r = recs + (size_t)g * 4;
        r[0] = kmin;
        r[1] = ((unsigned long long)scnt << 32) | sfirst;
        r[2] = scnt ? tbits(ncol[sfirst]) : 0ull;
        red_add_release(cnt, 1u);
        *s_ok = (int)wait_ctr(cnt, target, err, spin_limit);
    }
    named_sync(2, NT);
    if (!*s_ok) {
        out.status = ST_TIMEOUT;
        return out;
    }
    // every slice's record, in one batch of loads
    unsigned long long kk[R], fc[R];
    unsigned long long lk = ~0ull;
#pragma unroll
    for (int u = 0; u < R; ++u) {
        const int k = stid + u * NT;
        kk[u] = k < G ? __ldcg(recs + (size_t)k * 4) : ~0ull;
        fc[u] = k < G ? __ldcg(recs + (size_t)k * 4 + 1) : 0ull;
        if (k < G) vtab[k] = __ldcg(recs + (size_t)k * 4 + 2);
        lk = kk[u] < lk ? kk[u] : lk;
    }
    const unsigned long long rstar = sel_min_u64<SW>(lk, selq);
    if (rstar == ~0ull) {
        out.status = ST_UNBOUNDED;
        return out;
    }
    const unsigned long long thr = screen_thr(rstar, (T)0);
    unsigned a = 0xffffffffu, b = 0;
#pragma unroll
    for (int u = 0; u < R; ++u)
        if (kk[u] <= thr) {
            const unsigned f = (unsigned)(fc[u] & 0xffffffffull);
            a = f < a ? f : a;
            b += (unsigned)(fc[u] >> 32);
        }
    unsigned wfirst, wcnt;
    sel_min_sum<SW>(a, b, sela, selb, &wfirst, &wcnt);  // its barriers also publish vtab
    out.key = rstar;
    if (wcnt == 1) {
        out.row = (int)wfirst;
        out.val = vtab[wfirst / (unsigned)rs];
    }
    return out;
}

// The exact round after near ties: each CTA's best exact candidate (rc, with
// the new column's entry at its row) goes through one more exchange; every CTA
// gets the winner and its entry.  slot: this round's records (xsel + G) and
// values (xval + G * kBlkVals).
template <typename T, int SW>
__device__ Cand ratio_exact(Cand rc, unsigned long long rcval, Cand *xsel, unsigned long long *xval,
                            unsigned *cnt, unsigned target, int *err, long long spin_limit, int G,
                            int g, int stid, Cand *selc, unsigned long long *selq,
                            unsigned long long *tab, volatile int *s_ok, unsigned long long *val,
                            int *status) {
    constexpr int NT = 32 * SW;
    if (stid == 0) {
        xsel[g] = rc;
        xval[(size_t)g * kBlkVals] = rcval;
        red_add_release(cnt, 1u);
        *s_ok = (int)wait_ctr(cnt, target, err, spin_limit);
    }
    named_sync(2, NT);
    if (!*s_ok) {
        *status = ST_TIMEOUT;
        return cand_empty();
    }
    unsigned long long k;
    const Cand e = scan_records_tab<NT, 1>(xsel, xval, G, stid, &k, tab);
    const Cand w = sel_min<SW>(e, k, selc, selq, &k);
    *val = tab[k];
    return w;
}

// x after the pass's pivots 0..np-1, for row i (pv: their pivot-row values at
// the column of x).
template <typename T>
__device__ __forceinline__ T blk_apply(T x, int i, int np, const int *pp, const T *const *pc,
                                       const T *pv) {
#pragma unroll
    for (int k = 0; k < kBlk; ++k)
        if (k < np) x = (i == pp[k]) ? pv[k] : tfma(-pc[k][i], pv[k], x);
    return x;
}

template <typename T, int SW, bool DIST, bool SKIP, int MAXT = kMaxThreads>
__global__ void __launch_bounds__(MAXT, 1)
    pivot_block_kernel(LpDesc *__restrict__ d, int W, int split, long long spin_limit,
                       long long budget) {
    typedef typename Vec<T>::type V;
    constexpr int VW = Vec<T>::W;
    constexpr int kSelThreads = 32 * SW;
    // values of a pricing record kept in shared memory: the pivot-row values
    // (np for record a, np + 1 for record b) and, with SKIP, the buffer bit
    constexpr int NVA = SKIP ? kRecTab : kBlk, NVB = SKIP ? kRecTab : kBlk + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Cand rbuf[2][32];
    __shared__ unsigned long long ubuf[32];
    __shared__ Cand wpart[32];
    __shared__ Cand selc[SW];
    __shared__ unsigned long long selq[SW];
    __shared__ unsigned sela[SW], selb[SW];
    __shared__ int s_flag, s_status, s_sok, s_uok, s_np, s_pend, s_abort;
    __shared__ volatile int s_zready;  // passes whose objective-row strip is in sz
    __shared__ int s_p[kBlk], s_q[kBlk], s_rz[kBlk];
    __shared__ unsigned long long s_tab[kMaxRecs * kRecTab];  // the records' values
    __shared__ unsigned short s_vl[kMaxThreads];     // the vectors updated this pass, in order
    __shared__ unsigned char s_res[2][kMaxThreads];  // buffer holding each vector's rows, by pass parity
    __shared__ unsigned char s_nz[kMaxThreads];      // the vector's rows may hold a -0
    __shared__ int s_cf[32], s_rowner;
    // balanced ownership (below): the slack vectors no CTA owns yet (a bit
    // each), every CTA's vector count, this CTA's slack-run vectors (global
    // vector indices) in the order it took them, and the leaving variables of
    // the next pass's pivots
    constexpr int kDynWords = SKIP ? 512 : 1, kDynG = SKIP ? 256 : 1;
    __shared__ unsigned s_unown[kDynWords];
    __shared__ unsigned short s_load[kDynG];
    __shared__ unsigned short s_ov[SKIP ? kMaxThreads : 1];
    __shared__ int s_nown, s_unc, s_lv[kBlk];

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
    const int NU = B - kSelThreads;
    const int lane = tid & 31;
    const bool selw = tid >= NU;
    const int stid = tid - NU;
    T *bufs[2] = {reinterpret_cast<T *>(d->T), reinterpret_cast<T *>(d->T2)};
    int cur = 0;
    const long long P = d->P;
    const int m = d->m, M = d->M, N = d->N;
    int *__restrict__ basis = d->basis;
    const int bland_after = d->bland_after;
    const unsigned long long lim_p = okey((T)d->eps_p);
    const unsigned long long lim_d = okey((T)(-d->eps_d));
    const unsigned long long zero_k = okey((T)0);
    long long iters = d->iters;
    const long long iter_limit =
        iters > 0x3fffffffffffffffll - budget ? 0x3fffffffffffffffll : iters + budget;
    int deg = d->deg;
    int status = ST_RUNNING;
    // pcnt counts pricing records; scnt counts selections done (the first
    // selection, then one per pass), after which the CTA reads no more of the
    // pass's source tableau
    unsigned *pcnt = d->bar + 64, *scnt = d->bar + 160;

    // The CTA's columns (local l <-> global gcol(l)), vpr vectors of VW
    // columns; the rhs column's local index here (or -1) and its CTA.
    //
    // Vectors left in place (SKIP, with split runs): the constraint rows of a vector live in
    // one of the two buffers, s_res[parity of the pass][vector].  A pass
    // updates a vector from that buffer into the other one, except a vector
    // whose entries in both pivot rows of the pass are zeros: Step 5 leaves
    // it as it is, bit for bit (fma(-c, +-0, t) = t for finite c and t not
    // -0, and the pivot row's entry pr = +0 / positive pivot = +0 is the one
    // there), so its rows stay where they are.  That holds while no
    // constraint row holds a -0 (the primal form's pivots are positive, so a
    // -0 comes only from the data or from an update rounding to -0, which
    // marks the vector in s_nz and the LP in d->negz; with d->negz set, the
    // launch starts by marking the vectors that hold one) and the pass's
    // pivot columns are finite.  Readers of a column take its buffer from s_res
    // (this CTA's columns) or from the record that named the column.  The
    // objective row follows the pass parity.
    //
    // Balanced ownership (SKIP, on a launch from the slack basis with no -0
    // anywhere: d->iters == 0 and !d->negz).  A slack column whose variable
    // is basic is an exact unit vector e_r with a zero objective entry, and a
    // pivot leaves it as it is unless its row r is the pivot row, that is
    // unless its variable leaves; so a vector of VW slack columns that are all
    // basic is left in place until one of them leaves.  Those vectors belong
    // to no CTA at first; when one of its variables leaves (every CTA knows
    // the leaving variables, from the selection), the vector goes to the CTA
    // with the fewest vectors (ties: the lowest index) for the rest of the
    // launch, so no vector changes hands and the CTAs' update work stays
    // within a vector of each other, where fixed runs give each CTA the
    // leaving slacks that happen to fall in its run.  Each CTA keeps its run
    // of structural columns; the other vectors of the slack run (structural,
    // rhs and padding columns) are dealt out the same way at the start.  All
    // CTAs make the same choices from the same data.  A pass with a
    // non-finite pivot-column entry gives out every vector left.
    constexpr int kSector = 32 / (int)sizeof(T);
    const Strip S = make_strip(g, G, W, split, P, kSector);
    const int vpa = S.wa / VW;  // the CTA's structural vectors
    // the slack vectors that may start unowned: [dv0, dv1)
    const int nst = N - 1 - m;  // structural columns
    const int dv0 = (nst + VW - 1) / VW, dv1 = (nst + m) / VW, vtot = (int)(P / VW);
    const int capv = W / VW;  // most vectors a CTA may own (its shared memory holds W columns)
    const bool dyn = SKIP && split > 0 && d->iters == 0 && !d->negz && G <= kDynG &&
                     dv1 - dv0 <= 32 * kDynWords && vtot < 65536 && capv <= kMaxThreads;
    int ws = S.w();
    int vpr = ws / VW;
    int rl = S.lcol(N - 1);
    // without SKIP the strip is the contiguous one: the mappings simplify
    auto gcol = [&](int l) -> int {
        if (!SKIP || l < S.wa) return S.a0 + l;
        if (!dyn) return S.b0 + (l - S.wa);
        const int k = l - S.wa;
        return (int)s_ov[k / VW] * VW + k % VW;
    };
    // (this CTA's columns only; -1 elsewhere)
    auto lcol = [&](int j) -> int {
        if (!SKIP) return j - S.a0;
        if (!dyn) return S.lcol(j);
        if ((unsigned)(j - S.a0) < (unsigned)S.wa) return j - S.a0;
        for (int k = 0; k < vpr - vpa; ++k)
            if ((int)s_ov[k] == j / VW) return S.wa + k * VW + j % VW;
        return -1;
    };
    // warp 0: vector v to the CTA with the fewest vectors below capv
    auto assign = [&](int v) {
        unsigned best = 0xffffffffu;
        for (int c = lane; c < G; c += 32) {
            const unsigned l = s_load[c];
            if (l < (unsigned)capv) best = min(best, (l << 16) | (unsigned)c);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) {
            if (best == 0xffffffffu) {  // never: the host leaves every CTA room
                atomicExch(d->err, 1);
            } else {
                const int c = (int)(best & 0xffffu);
                s_load[c] = (unsigned short)(s_load[c] + 1);
                if (c == g) {
                    s_ov[s_nown++] = (unsigned short)v;
                    // the objective row follows the pass parity for the CTA's
                    // vectors; this one's entries are still in the first buffer
                    if (cur != 0)
                        for (int k = 0; k < VW; ++k)
                            bufs[cur][(long long)m * P + (long long)v * VW + k] =
                                bufs[0][(long long)m * P + (long long)v * VW + k];
                }
                if (v == (N - 1) / VW) s_rowner = c;
            }
        }
        __syncwarp();
    };
    if constexpr (SKIP) {
        for (int v = tid; v < (dyn ? capv : vpr); v += B) {
            s_res[0][v] = 0;
            s_res[1][v] = 0;
            s_nz[v] = 0;
        }
        if (dyn) {
            for (int c = tid; c < G; c += B) s_load[c] = (unsigned short)(make_strip(c, G, W, split, P, kSector).wa / VW);
            for (int w = tid; w < kDynWords; w += B) {
                const int b0 = 32 * w, nb = dv1 - dv0 - b0;
                s_unown[w] = nb >= 32 ? 0xffffffffu : nb > 0 ? (1u << nb) - 1u : 0u;
            }
            if (tid == 0) {
                s_nown = 0;
                s_unc = dv1 - dv0;
                s_lv[0] = s_lv[1] = -1;
            }
            __syncthreads();
            if (tid < 32)  // the slack run's vectors that are not all slack columns
                for (int v = split / VW; v < vtot; ++v)
                    if (v < dv0 || v >= dv1) assign(v);
            __syncthreads();
            vpr = vpa + s_nown;
            ws = vpr * VW;
            rl = lcol(N - 1);
        }
        if (d->negz) {
            // a constraint row may hold a -0 (from the data, Phase I, an FP32
            // refresh or an earlier launch): mark the vectors that do, one
            // read of the CTA's columns
            __syncthreads();
            const int rows = B / vpr, v = tid % vpr, r0 = tid / vpr;
            if (r0 < rows) {
                const T *col = bufs[0] + gcol(v * VW);
                bool f = false;
                for (int i = r0; i < m; i += rows) f |= has_negzero(ldv(reinterpret_cast<const V *>(col + (long long)i * P)));
                if (f) s_nz[v] = 1;
            }
        }
    }
    if (tid == 0 && !dyn) {
        int o = 0;
        for (int k = 0; k < G; ++k)
            if (make_strip(k, G, W, split, P, kSector).lcol(N - 1) >= 0) {
                o = k;
                break;
            }
        s_rowner = o;
    }
    // shared memory: the pass's pivot rows on the strip, the objective row of
    // T2 on the strip, pivot a's row on the strip; scratch (shared or this
    // CTA's global slice): four pivot columns (this pass's two, the next
    // pass's two), the rhs column of the pass's source tableau (kept from
    // pass to pass, so the selection never reads it from the tableau),
    // screening keys
    const size_t wbytes = ((size_t)W * sizeof(T) + 15) & ~(size_t)15;
    T *sprow[kBlk] = {reinterpret_cast<T *>(smem_raw), reinterpret_cast<T *>(smem_raw + wbytes)};
    T *sz = reinterpret_cast<T *>(smem_raw + 2 * wbytes);
    T *spa = reinterpret_cast<T *>(smem_raw + 3 * wbytes);
    unsigned char *sc = d->scratch_stride > 0
                            ? reinterpret_cast<unsigned char *>(d->scratch) +
                                  (size_t)g * (size_t)d->scratch_stride
                            : smem_raw + 4 * wbytes;
    const size_t cbytes = ((size_t)M * sizeof(T) + 15) & ~(size_t)15;
    T *scol[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) scol[k] = reinterpret_cast<T *>(sc + k * cbytes);
    T *srhs = reinterpret_cast<T *>(sc + 4 * cbytes);
    unsigned long long *srk = reinterpret_cast<unsigned long long *>(sc + 5 * cbytes);
    // the distributed ratio test: this CTA's rows [r0, r1), the global slots
    // of the four pivot columns (as scol), the ratio records and the records
    // of the exact rounds (by parity of their counts), and their counters
    const int rsl = m > 0 ? (m + G - 1) / G : 1;
    const int r0 = min(m, g * rsl), r1 = min(m, r0 + rsl);
    const int ra0 = DIST ? r0 : 0, ra1 = DIST ? r1 : m;  // the rows this CTA forms
    T *gcs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        gcs[k] = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(d->colx) + k * cbytes);
    unsigned long long *rrec = d->part_vals + (size_t)32 * G;  // 2 x G x 4
    Cand *xsel = reinterpret_cast<Cand *>(d->part_vals + (size_t)48 * G);  // 2 x G
    unsigned long long *xval = d->part_vals + (size_t)52 * G;  // 2 x G x kBlkVals
    unsigned *rrcnt = d->bar + 192, *xcnt = d->bar + 224;
    unsigned nrr = 0, nx = 0;  // ratio rounds and exact rounds so far (the same in every CTA)
    const bool smem_scr = d->scratch_stride == 0;

    // ---- selection of the first pivot from the current tableau (all threads) ----
    int p = -1, q = -1;
    {
        const T *Tab = bufs[0];
        const int bland = deg >= bland_after;
        Cand c = cand_empty();
        const T *z = Tab + (long long)m * P;
        for (int l = tid; l < ws; l += B) {
            const int j = gcol(l);
            if (j >= N - 1) continue;
            const unsigned long long zk = okey(lds(z + j));
            if (zk < lim_d) cand_take(c, bland ? zero_k : zk, j, j);
        }
        c = block_min_c(c, rbuf[0]);
        // in the slots of pass 1's first records: pass 0 writes its records
        // while slower CTAs may still read these, pass 1 only after every
        // CTA's pass-0 selection, which follows this one
        if (tid == 0) d->part_sel[2 * G + g] = c;
        if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) status = ST_TIMEOUT;
        if (status == ST_RUNNING) {
            const Cand sel = load_partials_min(d->part_sel + 2 * G, G, rbuf[1]);
            if (sel.idx < 0) status = ST_OPTIMAL;
            else if (iters >= iter_limit) status = ST_ITER_LIMIT;
            else if (sel.idx >= N - 1) status = ST_TIMEOUT;  // never: a partial from outside the row
            else q = sel.idx;
        }
        if (status == ST_RUNNING) {
            unsigned long long lmin = ~0ull;
            for (int i = tid; i < M; i += B) {
                const T a = lds(Tab + (long long)i * P + q);
                scol[0][i] = a;
                if (i < m) {
                    const T rhs = lds(Tab + (long long)i * P + (N - 1));
                    const unsigned long long rk =
                        okey(a) > lim_p ? screen_key(pos_part(rhs), a) : ~0ull;
                    srhs[i] = rhs;
                    srk[i] = rk;
                    lmin = rk < lmin ? rk : lmin;
                }
            }
            const unsigned long long rstar = block_min_u(lmin, ubuf);
            if (rstar == ~0ull) {
                status = ST_UNBOUNDED;
            } else {
                const unsigned long long thr = screen_thr(rstar, (T)0);
                Cand rc = cand_empty();
                for (int i = tid; i < m; i += B)
                    if (srk[i] <= thr)
                        cand_take(rc, okey(pos_part(srhs[i]) / scol[0][i]), bland ? __ldcg(basis + i) : i, i);
                rc = block_min_c(rc, rbuf[0]);
                p = rc.idx;
                deg = (rc.vk == zero_k) ? deg + 1 : 0;
            }
        }
    }

    // the pass's pivots; pend: the status to report after this pass, when the
    // selection during the previous pass already ended the solve
    int np = 1, pend = ST_RUNNING;
    int pp[kBlk] = {p, -1}, qq[kBlk] = {q, -1};
    int cb = 0;          // the pass's pivot columns are scol[cb], scol[cb + 1] (mod 4)
    unsigned lk = 0;     // passes made in this launch
    if (tid == 0) s_zready = 0;
    if (tid == 0 && dyn && p >= 0) s_lv[0] = __ldcg(basis + p);  // the first pivot's leaving variable
    __syncthreads();
    if (tid == 0 && status != ST_TIMEOUT) red_add_release(scnt, 1u);  // the first selection
    while (status == ST_RUNNING) {
        if constexpr (SKIP) {
            if (dyn) {
                // the pass's leaving slack vectors go to their owners (with a
                // non-finite pivot-column entry, every vector still unowned:
                // the pass updates them all)
                const T *c0 = scol[cb], *c1 = scol[(cb + 1) & 3];
                int nf = 0;
                for (int i = tid; i < m; i += B)
                    nf |= (int)not_finite(c0[i]) | (int)(np > 1 && not_finite(c1[i]));
                nf = __syncthreads_or(nf);
                if (tid < 32) {
                    if (nf) {
                        for (int w = 0; w < kDynWords; ++w) {
                            unsigned bits = s_unown[w];
                            while (bits) {
                                const int b = __ffs(bits) - 1;
                                bits &= bits - 1u;
                                assign(dv0 + 32 * w + b);
                            }
                            __syncwarp();
                            if (lane == 0) s_unown[w] = 0u;
                        }
                        if (lane == 0) s_unc = 0;
                    } else {
                        for (int k = 0; k < np; ++k) {
                            const int lv = s_lv[k];
                            const int v = lv >= nst && lv < nst + m ? lv / VW : -1;
                            if (v >= dv0 && v < dv1) {
                                const int b = v - dv0;
                                if ((s_unown[b >> 5] >> (b & 31)) & 1u) {
                                    __syncwarp();
                                    if (lane == 0) {
                                        s_unown[b >> 5] &= ~(1u << (b & 31));
                                        --s_unc;
                                    }
                                    __syncwarp();
                                    assign(v);
                                }
                            }
                        }
                    }
                }
                __syncthreads();
                vpr = vpa + s_nown;
                ws = vpr * VW;
            }
        }
        const int ab = tid == 0 ? abort_peek(d->abort) : 0;  // used at the pass's end
        const T *A = bufs[cur];
        T *Bn = bufs[cur ^ 1];
        const T *pc[kBlk] = {scol[cb], scol[(cb + 1) & 3]};
        T *nc[kBlk] = {scol[(cb + 2) & 3], scol[(cb + 3) & 3]};
        T *gnc[kBlk] = {gcs[(cb + 2) & 3], gcs[(cb + 3) & 3]};
        const int par = lk & 1;
        Cand *recA = d->part_sel + (2 * par) * G, *recB = d->part_sel + (2 * par + 1) * G;
        unsigned long long *valA = d->part_vals + (size_t)(2 * par) * G * kBlkVals;
        unsigned long long *valB = d->part_vals + (size_t)(2 * par + 1) * G * kBlkVals;
        const unsigned tA = (unsigned)G * (2u * lk + 1u), tB = (unsigned)G * (2u * lk + 2u);
        const int nbland = deg >= bland_after;  // rule of pivot a's selection
        const bool select = pend == ST_RUNNING;
        if (!selw) {
            // the strip of the objective row is loaded with the pivot rows'
            V zt;
            if (tid < vpr) zt = ldv(reinterpret_cast<const V *>(A + (long long)m * P + gcol(tid * VW)));
            // Step 4 for the pass's pivots on this CTA's strip
            for (int l = tid; l < ws; l += NU) {
                const int j = gcol(l);
                const T *Ar = SKIP ? bufs[s_res[par][l / VW]] : A;
                const T r = lds(Ar + (long long)pp[0] * P + j) / pc[0][pp[0]];
                sprow[0][l] = r;
                if (np > 1) {
                    const T t = (pp[1] == pp[0]) ? r
                                                 : tfma(-pc[0][pp[1]], r, lds(Ar + (long long)pp[1] * P + j));
                    sprow[1][l] = t / pc[1][pp[1]];
                }
            }
            // a non-finite entry in a pivot column: update every vector
            int bad = 0;
            if constexpr (SKIP) {
                for (int i = tid; i < m; i += NU)
                    bad |= (int)not_finite(pc[0][i]) | (int)(np > 1 && not_finite(pc[1][i]));
                bad = named_bar_or(1, NU, bad);
            } else {
                named_sync(1, NU);
            }
            // the new strip of the objective row of T2, and the CTA's pricing record a
            Cand c = cand_empty();
            if (tid < vpr) {
#pragma unroll
                for (int k = 0; k < kBlk; ++k)
                    if (k < np) vfma(zt, pc[k][m], *reinterpret_cast<const V *>(sprow[k] + tid * VW));
                *reinterpret_cast<V *>(sz + tid * VW) = zt;
#pragma unroll
                for (int k = 0; k < VW; ++k) {
                    const int j = gcol(tid * VW) + k;
                    const unsigned long long zk = okey(getc(zt, k));
                    if (j < N - 1 && zk < lim_d) cand_take(c, nbland ? zero_k : zk, j, j);
                }
            }
            // vector tid is updated this pass (else both pivot rows are zero on it)
            bool fv = true;
            unsigned bfv = 0u;
            if constexpr (SKIP) {
                if (tid < vpr)
                    fv = bad || s_nz[tid] ||
                         !(zero_vec(*reinterpret_cast<const V *>(sprow[0] + tid * VW)) &&
                           (np < 2 || zero_vec(*reinterpret_cast<const V *>(sprow[1] + tid * VW))));
                else
                    fv = false;
                bfv = __ballot_sync(0xffffffffu, fv);
            }
            c = warp_min(c);
            if (lane == 0) {
                wpart[tid >> 5] = c;
                if constexpr (SKIP) s_cf[tid >> 5] = __popc(bfv);
            }
            named_sync(1, NU);
            if (tid < 32) {
                const Cand e = tid < NU / 32 ? wpart[tid] : cand_empty();
                const Cand r = warp_min(e);
                if (tid == 0) {
                    if (select) {
                        recA[g] = r;
                        unsigned long long *v = valA + (size_t)g * kBlkVals;
                        for (int k = 0; k < np; ++k) {
                            v[k] = r.idx >= 0 ? tbits(sprow[k][lcol(r.idx)]) : 0ull;
                            v[4 + k] = rl >= 0 ? tbits(sprow[k][rl]) : 0ull;
                        }
                        if constexpr (SKIP) v[3] = r.idx >= 0 ? s_res[par][lcol(r.idx) / VW] : 0ull;
                        red_add_release(pcnt, 1u);
                    }
                    __threadfence_block();
                    s_zready = (int)(lk + 1);  // sz, sprow of this pass ready for the selection
                    // This pass writes the previous pass's source: every CTA's
                    // selections so far must be done reading it (and the
                    // basis, whose entries for this pass's pivots CTA 0 writes
                    // now: this pass's selection never reads them, the next
                    // pass's reads them after this CTA's next record).  The
                    // wait overlaps the selection of this pass, which needs
                    // only the records.
                    const int ok = (int)wait_ctr(scnt, (unsigned)G * (lk + 1u), d->err, spin_limit);
                    if (ok && g == 0) {
                        for (int k = 0; k < np; ++k) {
                            if (iters + k < d->trace_cap) {
                                d->trace[2 * (iters + k)] = pp[k];
                                d->trace[2 * (iters + k) + 1] = qq[k];
                            }
                            basis[pp[k]] = qq[k];
                        }
                        d->last_p = pp[np - 1];
                        d->last_q = qq[np - 1];
                    }
                    s_uok = ok;
                }
            }
            // the updated vectors in order, nF of them (after the record: it
            // is on the selection's path, this is not)
            int nF = vpr;
            if constexpr (SKIP) {
                int of = 0;
                nF = 0;
                for (int w = 0; w < (NU >> 5); ++w) {
                    const int f = s_cf[w];
                    of += w < (tid >> 5) ? f : 0;
                    nF += f;
                }
                if (fv) s_vl[of + __popc(bfv & ((1u << lane) - 1u))] = (unsigned short)tid;
            }
            named_sync(1, NU);
            if (s_uok && tid < vpr) {
                *reinterpret_cast<V *>(Bn + (long long)m * P + gcol(tid * VW)) = zt;
                if constexpr (SKIP) s_res[par ^ 1][tid] = s_res[par][tid] ^ (fv ? 1 : 0);
            }
            if (s_uok && tid == 0 && d->work) {  // vectors x pivots updated and left in place
                atomicAdd(d->work, (unsigned long long)(nF * np));
                atomicAdd(d->work + 1, (unsigned long long)((vpr - nF + (dyn && g == 0 ? s_unc : 0)) * np));
            }
            // Step 5 for the pass's pivots on the constraint rows of the
            // updated vectors, every update thread on one of them
            const int rpp = nF > 0 ? NU / nF : 0;
            const int lr = nF > 0 ? tid / nF : 0;
            if (s_uok && lr < rpp) {
                const int lv = SKIP ? (int)s_vl[tid - lr * nF] : tid - lr * nF;
                const int rs = SKIP ? (int)s_res[par][lv] : cur;
                const int col0 = gcol(lv * VW);
                const T *abase = bufs[rs] + col0;
                T *bbase = bufs[rs ^ 1] + col0;
                const V pr0 = *reinterpret_cast<const V *>(sprow[0] + lv * VW);
                const int p0 = pp[0];
                const T *__restrict__ c0p = pc[0];
                bool nz = false;
                int i = lr;
                if (np == 2) {
                    const V pr1 = *reinterpret_cast<const V *>(sprow[1] + lv * VW);
                    const int p1 = pp[1];
                    const T *__restrict__ c1p = pc[1];
                    for (; i + 3 * rpp < m; i += 4 * rpp) {
                        const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                        V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                        V t1 = ldv(reinterpret_cast<const V *>(abase + (long long)i1 * P));
                        V t2 = ldv(reinterpret_cast<const V *>(abase + (long long)i2 * P));
                        V t3 = ldv(reinterpret_cast<const V *>(abase + (long long)i3 * P));
                        t0 = pivot_vec<T>(pivot_vec<T>(t0, i, p0, c0p[i], pr0), i, p1, c1p[i], pr1);
                        t1 = pivot_vec<T>(pivot_vec<T>(t1, i1, p0, c0p[i1], pr0), i1, p1, c1p[i1], pr1);
                        t2 = pivot_vec<T>(pivot_vec<T>(t2, i2, p0, c0p[i2], pr0), i2, p1, c1p[i2], pr1);
                        t3 = pivot_vec<T>(pivot_vec<T>(t3, i3, p0, c0p[i3], pr0), i3, p1, c1p[i3], pr1);
                        if constexpr (SKIP) nz |= has_negzero(t0) | has_negzero(t1) | has_negzero(t2) | has_negzero(t3);
                        *reinterpret_cast<V *>(bbase + (long long)i * P) = t0;
                        *reinterpret_cast<V *>(bbase + (long long)i1 * P) = t1;
                        *reinterpret_cast<V *>(bbase + (long long)i2 * P) = t2;
                        *reinterpret_cast<V *>(bbase + (long long)i3 * P) = t3;
                    }
                    for (; i < m; i += rpp) {
                        V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                        t0 = pivot_vec<T>(pivot_vec<T>(t0, i, p0, c0p[i], pr0), i, p1, c1p[i], pr1);
                        if constexpr (SKIP) nz |= has_negzero(t0);
                        *reinterpret_cast<V *>(bbase + (long long)i * P) = t0;
                    }
                } else {
                    for (; i + 3 * rpp < m; i += 4 * rpp) {
                        const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                        V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                        V t1 = ldv(reinterpret_cast<const V *>(abase + (long long)i1 * P));
                        V t2 = ldv(reinterpret_cast<const V *>(abase + (long long)i2 * P));
                        V t3 = ldv(reinterpret_cast<const V *>(abase + (long long)i3 * P));
                        t0 = pivot_vec<T>(t0, i, p0, c0p[i], pr0);
                        t1 = pivot_vec<T>(t1, i1, p0, c0p[i1], pr0);
                        t2 = pivot_vec<T>(t2, i2, p0, c0p[i2], pr0);
                        t3 = pivot_vec<T>(t3, i3, p0, c0p[i3], pr0);
                        if constexpr (SKIP) nz |= has_negzero(t0) | has_negzero(t1) | has_negzero(t2) | has_negzero(t3);
                        *reinterpret_cast<V *>(bbase + (long long)i * P) = t0;
                        *reinterpret_cast<V *>(bbase + (long long)i1 * P) = t1;
                        *reinterpret_cast<V *>(bbase + (long long)i2 * P) = t2;
                        *reinterpret_cast<V *>(bbase + (long long)i3 * P) = t3;
                    }
                    for (; i < m; i += rpp) {
                        V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                        t0 = pivot_vec<T>(t0, i, p0, c0p[i], pr0);
                        if constexpr (SKIP) nz |= has_negzero(t0);
                        *reinterpret_cast<V *>(bbase + (long long)i * P) = t0;
                    }
                }
                if (SKIP && nz) {  // this vector is never left in place again, nor any later
                    s_nz[lv] = 1;
                    d->negz = 1;
                }
            }
        } else {
            // selection of the next pass's pivots a and b
            int st = ST_RUNNING, nnp = 0, npend = ST_RUNNING;
            int pa = -1, qa = -1, pb = -1, qb = -1, rza = 0, rzb = 0;
            T piva = (T)0;  // pivot a's entry of its column
            // the basic variable of row i after the pass's pivots
            auto bkey = [&](int i) -> int {
                if (np > 1 && i == pp[1]) return qq[1];
                if (i == pp[0]) return qq[0];
                return __ldcg(basis + i);
            };
            const T *colA = nc[0];
            if (!select) {
                st = pend;  // the previous pass's selection already ended the solve
            } else {
                // ---- pivot a (Step 2): the pricing records of this pass ----
                if (stid == 0) s_sok = (int)wait_ctr(pcnt, tA, d->err, spin_limit);
                named_sync(2, kSelThreads);
                unsigned long long ka = 0ull;
                unsigned long long rvb[kBlk];  // the rhs owner's values, loaded with the records
                if (!s_sok) {
                    st = ST_TIMEOUT;
                } else {
#pragma unroll
                    for (int k = 0; k < kBlk; ++k) rvb[k] = __ldcg(valA + (size_t)s_rowner * kBlkVals + 4 + k);
                    const Cand e = scan_records_tab<kSelThreads, NVA>(recA, valA, G, stid, &ka, s_tab);
                    const Cand sel = sel_min<SW>(e, ka, selc, selq, &ka);
                    if (sel.idx < 0) st = ST_OPTIMAL;
                    else if (iters + np >= iter_limit) st = ST_ITER_LIMIT;
                    else if (sel.idx >= N - 1) st = ST_TIMEOUT;  // never: a record from outside the row
                    else qa = sel.idx;
                    if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                }
                if (st == ST_RUNNING) {
                    // the pass's pivot-row values at q_a and at the rhs
                    T pvq[kBlk], pvr[kBlk];
#pragma unroll
                    for (int k = 0; k < kBlk; ++k) {
                        pvq[k] = tfrom<T>(s_tab[ka * NVA + k]);
                        pvr[k] = tfrom<T>(rvb[k]);
                    }
                    const T *Aq = SKIP ? bufs[s_tab[ka * NVA + 3] & 1] : A;  // column q_a's rows
                    // column q_a and rhs of T2 on this CTA's rows (Step 3,
                    // distributed); the rhs from the one of T0 kept in scratch,
                    // which becomes T2's
                    T *ncol = nc[0];
                    unsigned long long lmin = ~0ull;
                    // the objective row's entry rides with the first batch
                    const T am = stid == 0 ? lds(A + (long long)m * P + qa) : (T)0;
                    for (int i0 = ra0 + stid; i0 < ra1; i0 += kColRows * kSelThreads) {
                        T av[kColRows];
#pragma unroll
                        for (int u = 0; u < kColRows; ++u) {
                            const int i = i0 + u * kSelThreads;
                            av[u] = i < ra1 ? lds(Aq + (long long)i * P + qa) : (T)0;
                        }
#pragma unroll
                        for (int u = 0; u < kColRows; ++u) {
                            const int i = i0 + u * kSelThreads;
                            if (i >= ra1) break;
                            const T a = blk_apply<T>(av[u], i, np, pp, pc, pvq);
                            ncol[i] = a;
                            if (DIST) gnc[0][i] = a;
                            const T rhs = blk_apply<T>(srhs[i], i, np, pp, pc, pvr);
                            srhs[i] = rhs;
                            const unsigned long long rk =
                                okey(a) > lim_p ? screen_key(pos_part(rhs), a) : ~0ull;
                            srk[i] = rk;
                            lmin = rk < lmin ? rk : lmin;
                        }
                    }
                    if (stid == 0) {  // every CTA forms the objective row's entry itself
                        ncol[m] = blk_apply<T>(am, m, np, pp, pc, pvq);
                        if (DIST && g == 0) gnc[0][m] = ncol[m];
                    }
                    if constexpr (!DIST) {
                        // every row in this CTA: the screened test, exact on near ties
                        const unsigned long long rstar = sel_min_u64<SW>(lmin, selq);
                        if (rstar == ~0ull) {
                            st = ST_UNBOUNDED;
                        } else {
                            const unsigned long long thr = screen_thr(rstar, (T)0);
                            unsigned first = 0xffffffffu, cnt = 0;
                            for (int i = stid; i < m; i += kSelThreads)
                                if (srk[i] <= thr) {
                                    first = (unsigned)i < first ? (unsigned)i : first;
                                    ++cnt;
                                }
                            unsigned gfirst, gcnt;
                            sel_min_sum<SW>(first, cnt, sela, selb, &gfirst, &gcnt);
                            if (gcnt == 1) {
                                pa = (int)gfirst;
                                rza = srk[pa] == zero_k;
                            } else {
                                Cand rc = cand_empty();
                                for (int i = stid; i < m; i += kSelThreads)
                                    if (srk[i] <= thr) {
                                        const T nm = pos_part(srhs[i]);
                                        const unsigned long long vk =
                                            tbits(nm) == 0ull ? zero_k : okey(nm / ncol[i]);
                                        cand_take(rc, vk, nbland ? bkey(i) : i, i);
                                    }
                                rc = sel_min<SW>(rc, 0ull, selc, selq, nullptr);
                                pa = rc.idx;
                                rza = rc.vk == zero_k;
                            }
                            piva = ncol[pa];
                        }
                    } else {
                    const RatioPick rp = ratio_slices<T, SW>(
                        lmin, srk, ncol, r0, r1, rsl, rrec + (size_t)(nrr & 1) * G * 4, rrcnt,
                        (unsigned)G * (nrr + 1u), d->err, spin_limit, G, g, stid, selq, sela, selb,
                        s_tab, &s_sok);
                    ++nrr;
                    if (rp.status != ST_RUNNING) {
                        st = rp.status;
                    } else if (rp.row >= 0) {
                        pa = rp.row;
                        piva = tfrom<T>(rp.val);
                        rza = rp.key == zero_k;
                    } else {
                        // near ties: the exact quotients of the rows within the
                        // threshold, one more exchange
                        const unsigned long long thr = screen_thr(rp.key, (T)0);
                        Cand rc = cand_empty();
                        for (int i = r0 + stid; i < r1; i += kSelThreads)
                            if (srk[i] <= thr) {
                                const T nm = pos_part(srhs[i]);
                                const unsigned long long vk =
                                    tbits(nm) == 0ull ? zero_k : okey(nm / ncol[i]);
                                cand_take(rc, vk, nbland ? bkey(i) : i, i);
                            }
                        rc = sel_min<SW>(rc, 0ull, selc, selq, nullptr);
                        unsigned long long v;
                        const Cand w = ratio_exact<T, SW>(
                            rc, rc.idx >= 0 ? tbits(ncol[rc.idx]) : 0ull, xsel + (size_t)(nx & 1) * G,
                            xval + (size_t)(nx & 1) * G * kBlkVals, xcnt, (unsigned)G * (nx + 1u),
                            d->err, spin_limit, G, g, stid, selc, selq, s_tab, &s_sok, &v, &st);
                        ++nx;
                        pa = w.idx;
                        piva = tfrom<T>(v);
                        rza = w.vk == zero_k;
                    }
                    // the whole column q_a for the next pass's update, copied
                    // while pivot b is selected
                    if (st == ST_RUNNING) fill_column(ncol, gnc[0], cbytes, stid, kSelThreads, smem_scr);
                    }
                }
                if (st == ST_RUNNING) {
                    // ---- pivot b: pivot a's row on this strip, the objective row
                    // after pivot a, the CTA's pricing record b ----
                    const int nblandb = (rza ? deg + 1 : 0) >= bland_after;
                    if (stid == 0) {  // this pass's sprow and sz (written by the update warps)
                        const long long t0 = clock64();
                        int ok = 1;
                        while (s_zready < (int)(lk + 1)) {
                            if (clock64() - t0 > spin_limit || *(volatile int *)d->err) {
                                atomicExch(d->err, 1);
                                ok = 0;
                                break;
                            }
                        }
                        s_sok = ok;
                    }
                    named_sync(2, kSelThreads);
                    __threadfence_block();
                    if (!s_sok) {
                        st = ST_TIMEOUT;
                    } else {
                        Cand e = cand_empty();
                        for (int l = stid; l < ws; l += kSelThreads) {
                            const int j = gcol(l);
                            T r = lds((SKIP ? bufs[s_res[par][l / VW]] : A) + (long long)pa * P + j);
#pragma unroll
                            for (int k = 0; k < kBlk; ++k)
                                if (k < np)
                                    r = (pa == pp[k]) ? sprow[k][l] : tfma(-pc[k][pa], sprow[k][l], r);
                            const T pra = r / piva;
                            spa[l] = pra;
                            const unsigned long long zk = okey(tfma(-colA[m], pra, sz[l]));
                            if (j < N - 1 && zk < lim_d) cand_take(e, nblandb ? zero_k : zk, j, j);
                        }
                        e = sel_min<SW>(e, 0ull, selc, selq, nullptr);
                        if (stid == 0) {
                            recB[g] = e;
                            unsigned long long *v = valB + (size_t)g * kBlkVals;
                            for (int k = 0; k <= np; ++k) {
                                const T *row = k < np ? sprow[k] : spa;
                                v[k] = e.idx >= 0 ? tbits(row[lcol(e.idx)]) : 0ull;
                                v[4 + k] = rl >= 0 ? tbits(row[rl]) : 0ull;
                            }
                            if constexpr (SKIP) v[3] = e.idx >= 0 ? s_res[par][lcol(e.idx) / VW] : 0ull;
                            red_add_release(pcnt, 1u);
                        }
                        // ---- pivot b (Step 2): the pricing records ----
                        if (stid == 0) s_sok = (int)wait_ctr(pcnt, tB, d->err, spin_limit);
                        named_sync(2, kSelThreads);
                        unsigned long long kb = 0ull;
                        unsigned long long rvb[kBlk + 1];  // the rhs owner's values
                        if (!s_sok) {
                            st = ST_TIMEOUT;
                        } else {
#pragma unroll
                            for (int k = 0; k <= kBlk; ++k)
                                rvb[k] = __ldcg(valB + (size_t)s_rowner * kBlkVals + 4 + k);
                            const Cand f = scan_records_tab<kSelThreads, NVB>(recB, valB, G, stid, &kb, s_tab);
                            const Cand sel = sel_min<SW>(f, kb, selc, selq, &kb);
                            nnp = 1;
                            if (sel.idx < 0) npend = ST_OPTIMAL;
                            else if (iters + np + 1 >= iter_limit) npend = ST_ITER_LIMIT;
                            else if (sel.idx >= N - 1) st = ST_TIMEOUT;  // never
                            else qb = sel.idx;
                            if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                        }
                        if (st == ST_RUNNING && qb >= 0) {
                            T pvq[kBlk + 1], pvr[kBlk + 1];
#pragma unroll
                            for (int k = 0; k <= kBlk; ++k) {
                                pvq[k] = tfrom<T>(s_tab[kb * NVB + k]);
                                pvr[k] = tfrom<T>(rvb[k]);
                            }
                            const T *Aq = SKIP ? bufs[s_tab[kb * NVB + 3] & 1] : A;  // column q_b's rows
                            // column q_b and rhs after pivot a on this CTA's rows
                            // (Step 3, distributed); scratch keeps T2's rhs for the
                            // next pass
                            T *ncol = nc[1];
                            unsigned long long lmin = ~0ull;
                            const T am = stid == 0 ? lds(A + (long long)m * P + qb) : (T)0;
                            for (int i0 = ra0 + stid; i0 < ra1; i0 += kColRows * kSelThreads) {
                                T av[kColRows];
#pragma unroll
                                for (int u = 0; u < kColRows; ++u) {
                                    const int i = i0 + u * kSelThreads;
                                    av[u] = i < ra1 ? lds(Aq + (long long)i * P + qb) : (T)0;
                                }
#pragma unroll
                                for (int u = 0; u < kColRows; ++u) {
                                    const int i = i0 + u * kSelThreads;
                                    if (i >= ra1) break;
                                    const T ca = colA[i];
                                    T a = blk_apply<T>(av[u], i, np, pp, pc, pvq);
                                    a = (i == pa) ? pvq[np] : tfma(-ca, pvq[np], a);
                                    ncol[i] = a;
                                    if (DIST) gnc[1][i] = a;
                                    const T h = (i == pa) ? pvr[np] : tfma(-ca, pvr[np], srhs[i]);
                                    const unsigned long long rk =
                                        okey(a) > lim_p ? screen_key(pos_part(h), a) : ~0ull;
                                    srk[i] = rk;
                                    lmin = rk < lmin ? rk : lmin;
                                }
                            }
                            if (stid == 0) {  // pa < m
                                ncol[m] = tfma(-colA[m], pvq[np], blk_apply<T>(am, m, np, pp, pc, pvq));
                                if (DIST && g == 0) gnc[1][m] = ncol[m];
                            }
                            if constexpr (!DIST) {
                                const unsigned long long rstar = sel_min_u64<SW>(lmin, selq);
                                if (rstar == ~0ull) {
                                    npend = ST_UNBOUNDED;
                                } else {
                                    const unsigned long long thr = screen_thr(rstar, (T)0);
                                    unsigned first = 0xffffffffu, cnt = 0;
                                    for (int i = stid; i < m; i += kSelThreads)
                                        if (srk[i] <= thr) {
                                            first = (unsigned)i < first ? (unsigned)i : first;
                                            ++cnt;
                                        }
                                    unsigned gfirst, gcnt;
                                    sel_min_sum<SW>(first, cnt, sela, selb, &gfirst, &gcnt);
                                    if (gcnt == 1) {
                                        pb = (int)gfirst;
                                        rzb = srk[pb] == zero_k;
                                    } else {
                                        Cand rc = cand_empty();
                                        for (int i = stid; i < m; i += kSelThreads)
                                            if (srk[i] <= thr) {
                                                const T nm = pos_part((i == pa) ? pvr[np]
                                                                                : tfma(-colA[i], pvr[np], srhs[i]));
                                                const unsigned long long vk =
                                                    tbits(nm) == 0ull ? zero_k : okey(nm / ncol[i]);
                                                const int key = nblandb ? (i == pa ? qa : bkey(i)) : i;
                                                cand_take(rc, vk, key, i);
                                            }
                                        rc = sel_min<SW>(rc, 0ull, selc, selq, nullptr);
                                        pb = rc.idx;
                                        rzb = rc.vk == zero_k;
                                    }
                                    nnp = 2;
                                }
                            } else {
                            const RatioPick rp = ratio_slices<T, SW>(
                                lmin, srk, ncol, r0, r1, rsl, rrec + (size_t)(nrr & 1) * G * 4, rrcnt,
                                (unsigned)G * (nrr + 1u), d->err, spin_limit, G, g, stid, selq, sela,
                                selb, s_tab, &s_sok);
                            ++nrr;
                            if (rp.status == ST_TIMEOUT) {
                                st = ST_TIMEOUT;
                            } else if (rp.status == ST_UNBOUNDED) {
                                npend = ST_UNBOUNDED;
                            } else {
                                if (rp.row >= 0) {
                                    pb = rp.row;
                                    rzb = rp.key == zero_k;
                                } else {
                                    const unsigned long long thr = screen_thr(rp.key, (T)0);
                                    Cand rc = cand_empty();
                                    for (int i = r0 + stid; i < r1; i += kSelThreads)
                                        if (srk[i] <= thr) {
                                            const T nm = pos_part((i == pa) ? pvr[np]
                                                                            : tfma(-colA[i], pvr[np], srhs[i]));
                                            const unsigned long long vk =
                                                tbits(nm) == 0ull ? zero_k : okey(nm / ncol[i]);
                                            const int key = nblandb ? (i == pa ? qa : bkey(i)) : i;
                                            cand_take(rc, vk, key, i);
                                        }
                                    rc = sel_min<SW>(rc, 0ull, selc, selq, nullptr);
                                    unsigned long long v;
                                    const Cand w = ratio_exact<T, SW>(
                                        rc, rc.idx >= 0 ? tbits(ncol[rc.idx]) : 0ull,
                                        xsel + (size_t)(nx & 1) * G, xval + (size_t)(nx & 1) * G * kBlkVals,
                                        xcnt, (unsigned)G * (nx + 1u), d->err, spin_limit, G, g, stid,
                                        selc, selq, s_tab, &s_sok, &v, &st);
                                    ++nx;
                                    pb = w.idx;
                                    rzb = w.vk == zero_k;
                                }
                                if (st == ST_RUNNING) {
                                    fill_column(ncol, gnc[1], cbytes, stid, kSelThreads, smem_scr);
                                    nnp = 2;
                                }
                            }
                            }
                        }
                    }
                }
            }
            // the pass's pivot columns are copied in full before the next pass
            fill_wait();
            // every selection thread is done reading this pass's source
            named_sync(2, kSelThreads);
            if (stid == 0) {
                if (st != ST_TIMEOUT) red_add_release(scnt, 1u);
                s_status = st;
                s_np = nnp;
                s_pend = npend;
                s_p[0] = pa;
                s_q[0] = qa;
                s_p[1] = pb;
                s_q[1] = qb;
                s_rz[0] = rza;
                s_rz[1] = rzb;
                if constexpr (SKIP) {  // the leaving variables of the next pass's pivots
                    s_lv[0] = pa >= 0 ? bkey(pa) : -1;
                    s_lv[1] = pb >= 0 ? (pb == pa ? qa : bkey(pb)) : -1;
                }
            }
        }
        // the CTA's pass and its selection of the next pass are done
        if (tid == 0) {
            s_abort = ab;  // past the host's deadline: stop, and end every CTA's waits
            if (ab) atomicExch(d->err, 1);
        }
        __syncthreads();
        iters += np;
        ++lk;
        status = s_abort ? ST_TIMEOUT : s_status;
        if (!s_uok) status = ST_TIMEOUT;
        if (status == ST_RUNNING) {
            np = s_np;
            pend = s_pend;
            for (int k = 0; k < kBlk; ++k) {
                pp[k] = s_p[k];
                qq[k] = s_q[k];
            }
            deg = s_rz[0] ? deg + 1 : 0;
            if (np > 1) deg = s_rz[1] ? deg + 1 : 0;
            cb = (cb + 2) & 3;
        }
        cur ^= 1;
        // no grid barrier: a CTA starts the next pass as soon as its own is
        // done; the counters order everything that crosses CTAs
    }

    // Hand over one buffer: the rows of the vectors last left in the other
    // one are copied into it (the objective row is there already).  No
    // reader of the passes reads a vector from the buffer it is not in.
    if constexpr (SKIP) {
        const unsigned char *res = s_res[lk & 1];
        for (int v = 0; v < vpr; ++v) {
            if (res[v] == cur) continue;
            const T *src = bufs[res[v]] + gcol(v * VW);
            T *dst = bufs[cur] + gcol(v * VW);
            for (int i = tid; i < m; i += B)
                *reinterpret_cast<V *>(dst + (long long)i * P) = ldv(reinterpret_cast<const V *>(src + (long long)i * P));
        }
        if (dyn && cur != 0) {
            // the vectors no CTA took are in the first buffer, objective
            // entries included: CTA u mod G copies the u-th of them
            for (int w = 0; w < kDynWords; ++w) {
                unsigned bits = s_unown[w];
                while (bits) {
                    const int b = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    const int u = 32 * w + b;
                    if (u % G != g) continue;
                    const long long col = (long long)(dv0 + u) * VW;
                    for (int i = tid; i < M; i += B)
                        *reinterpret_cast<V *>(bufs[1] + (long long)i * P + col) =
                            ldv(reinterpret_cast<const V *>(bufs[0] + (long long)i * P + col));
                }
            }
        }
    }
    if (g == 0 && tid == 0) {
        // every CTA's last selection is done, and with it its last wait
        wait_ctr(scnt, (unsigned)G * (lk + 1u), d->err, spin_limit);
        d->status = (*(volatile int *)d->err) ? ST_TIMEOUT : status;
        d->iters = iters;
        d->iter_limit = iter_limit;
        d->deg = deg;
        d->T = bufs[cur];  // hand over the buffer holding the last tableau
        d->T2 = bufs[cur ^ 1];
    }
}

// ---------------------------------------------------------------------------
// Two pivots per pass for the dual form (dual simplex), double-buffered.
//
// The pass is the two-pivot primal kernel's (the same update warps' code:
// Step 4 for both pivots on the strip, then both elementary operations per
// element in order).  The selection warps choose the next two pivots from the
// pass's source buffer: leaving row r_a from the rhs of T2 (every CTA, all
// rows), row r_a of T2 on the CTA's strip and its dual ratio test, one
// record per CTA (with the pass's pivot-row values at its column) for the
// entering column q_a, column q_a of T2 (every CTA, all rows); then the rhs
// after pivot a (from values already in scratch), leaving row r_b, row r_b
// after pivot a on the strip, a second round of records for q_b, column q_b
// after pivot a.  As in the primal kernel, no grid barrier separates the
// passes: a counter of selections done guards the rewrite of the source.
template <typename T, int SW>
__global__ void __launch_bounds__(kMaxThreads, 1)
    pivot_block_dual_kernel(LpDesc *__restrict__ d, int W, long long spin_limit, long long budget) {
    typedef typename Vec<T>::type V;
    constexpr int VW = Vec<T>::W;
    constexpr int kSelThreads = 32 * SW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Cand rbuf[2][32];
    __shared__ Cand selc[SW];
    __shared__ unsigned long long selq[SW];
    __shared__ int s_flag, s_status, s_sok, s_uok, s_np, s_pend, s_abort;
    __shared__ volatile int s_zready;
    __shared__ int s_p[kBlk], s_q[kBlk], s_rz[kBlk];
    __shared__ unsigned long long s_tab[kMaxRecs * (kBlk + 1)];  // the records' values

    const int G = gridDim.x, g = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
    const int NU = B - kSelThreads;
    const int lane = tid & 31;
    const bool selw = tid >= NU;
    const int stid = tid - NU;
    T *bufs[2] = {reinterpret_cast<T *>(d->T), reinterpret_cast<T *>(d->T2)};
    int cur = 0;
    const long long P = d->P;
    const int m = d->m, M = d->M, N = d->N;
    int *__restrict__ basis = d->basis;
    const int bland_after = d->bland_after;
    const unsigned long long lim_np = okey((T)(-d->eps_p));
    const unsigned long long lim_r = okey((T)(-d->eps_r));
    const unsigned long long zero_k = okey((T)0);
    long long iters = d->iters;
    const long long iter_limit =
        iters > 0x3fffffffffffffffll - budget ? 0x3fffffffffffffffll : iters + budget;
    int deg = d->deg;
    int status = ST_RUNNING;
    // rcnt counts the records; scnt the selections done (the first, then one
    // per pass), as in the primal kernel
    unsigned *rcnt = d->bar + 128, *scnt = d->bar + 160;

    const int c0 = g * W;
    const int c1 = (int)min((long long)c0 + W, P);
    const int jend = min(c1, N - 1);
    const int vpr = (c1 - c0) / VW;
    const int rpp = NU / vpr;
    const int lr = tid / vpr, lv = tid - lr * vpr;
    const bool active = !selw && lr < rpp;
    const int col0 = c0 + lv * VW;
    // shared memory: the pass's pivot rows on the strip, the objective row of
    // T2 on the strip, row r_a of T2 on the strip; scratch: four pivot
    // columns, the rhs column of the pass's source tableau (kept from pass to
    // pass, so the selection never reads it from the tableau)
    const size_t wbytes = ((size_t)W * sizeof(T) + 15) & ~(size_t)15;
    T *sprow[kBlk] = {reinterpret_cast<T *>(smem_raw), reinterpret_cast<T *>(smem_raw + wbytes)};
    T *sz = reinterpret_cast<T *>(smem_raw + 2 * wbytes);
    T *sra = reinterpret_cast<T *>(smem_raw + 3 * wbytes);
    unsigned char *sc = d->scratch_stride > 0
                            ? reinterpret_cast<unsigned char *>(d->scratch) +
                                  (size_t)g * (size_t)d->scratch_stride
                            : smem_raw + 4 * wbytes;
    const size_t cbytes = ((size_t)M * sizeof(T) + 15) & ~(size_t)15;
    T *scol[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) scol[k] = reinterpret_cast<T *>(sc + k * cbytes);
    T *srhs = reinterpret_cast<T *>(sc + 4 * cbytes);

    // ---- the first pivot from the current tableau (all threads) ----
    int p = -1, q = -1;
    {
        const T *A = bufs[0];
        const int bland = deg >= bland_after;
        Cand c = cand_empty();
        for (int i = tid; i < m; i += B) {
            const T rhs = lds(A + (long long)i * P + (N - 1));
            srhs[i] = rhs;
            const unsigned long long vk = okey(rhs);
            if (vk < lim_r) cand_take(c, bland ? zero_k : vk, bland ? __ldcg(basis + i) : i, i);
        }
        c = block_min_c(c, rbuf[0]);
        if (c.idx < 0) status = ST_OPTIMAL;
        else if (iters >= iter_limit) status = ST_ITER_LIMIT;
        else p = c.idx;
        if (status == ST_RUNNING) {
            const T *rowr = A + (long long)p * P, *z = A + (long long)m * P;
            Cand e = cand_empty();
            for (int j = c0 + tid; j < jend; j += B) {
                const T a = lds(rowr + j);
                if (okey(a) < lim_np) cand_take(e, okey(pos_part(lds(z + j)) / neg(a)), j, j);
            }
            e = block_min_c(e, rbuf[1]);
            if (tid == 0) d->part_sel[2 * G + g] = e;
            if (!grid_sync(d->bar, d->err, G, spin_limit, &s_flag)) status = ST_TIMEOUT;
            if (status == ST_RUNNING) {
                const Cand sel = load_partials_min(d->part_sel + 2 * G, G, rbuf[0]);
                if (sel.idx < 0) {
                    status = ST_INFEASIBLE;
                } else if (sel.idx >= N - 1) {
                    status = ST_TIMEOUT;  // never: a partial from outside the row
                } else {
                    q = sel.idx;
                    deg = (sel.vk == zero_k) ? deg + 1 : 0;
                    for (int i = tid; i < M; i += B) scol[0][i] = lds(A + (long long)i * P + q);
                }
            }
        }
    }
    int np = 1, pend = ST_RUNNING;
    int pp[kBlk] = {p, -1}, qq[kBlk] = {q, -1};
    int npv = 0, ppv[kBlk] = {-1, -1}, qqv[kBlk] = {-1, -1};  // the previous pass's pivots
    int cb = 0;
    unsigned lk = 0;
    if (tid == 0) s_zready = 0;
    __syncthreads();
    if (tid == 0 && status != ST_TIMEOUT) red_add_release(scnt, 1u);  // the first selection

    while (status == ST_RUNNING) {
        const int ab = tid == 0 ? abort_peek(d->abort) : 0;  // used at the pass's end
        const T *A = bufs[cur];
        T *Bn = bufs[cur ^ 1];
        const T *pc[kBlk] = {scol[cb], scol[(cb + 1) & 3]};
        T *nc[kBlk] = {scol[(cb + 2) & 3], scol[(cb + 3) & 3]};
        const int par = lk & 1;
        Cand *recA = d->part_sel + (2 * par) * G, *recB = d->part_sel + (2 * par + 1) * G;
        unsigned long long *valA = d->part_vals + (size_t)(2 * par) * G * kBlkVals;
        unsigned long long *valB = d->part_vals + (size_t)(2 * par + 1) * G * kBlkVals;
        const unsigned tA = (unsigned)G * (2u * lk + 1u), tB = (unsigned)G * (2u * lk + 2u);
        (void)lane;
        const int nbland = deg >= bland_after;  // rule of pivot a's selection
        const bool select = pend == ST_RUNNING;
        if (!selw) {
            // the strip of the objective row is loaded with the pivot rows'
            V zt;
            if (tid < vpr) zt = ldv(reinterpret_cast<const V *>(A + (long long)m * P + c0 + tid * VW));
            // Step 4 for the pass's pivots on this CTA's strip
            for (int j = c0 + tid; j < c1; j += NU) {
                const T r = lds(A + (long long)pp[0] * P + j) / pc[0][pp[0]];
                sprow[0][j - c0] = r;
                if (np > 1) {
                    const T t = (pp[1] == pp[0]) ? r
                                                 : tfma(-pc[0][pp[1]], r, lds(A + (long long)pp[1] * P + j));
                    sprow[1][j - c0] = t / pc[1][pp[1]];
                }
            }
            named_sync(1, NU);
            // the new strip of the objective row of T2, also for the selection
            if (tid < vpr) {
#pragma unroll
                for (int k = 0; k < kBlk; ++k)
                    if (k < np) vfma(zt, pc[k][m], *reinterpret_cast<const V *>(sprow[k] + tid * VW));
                *reinterpret_cast<V *>(sz + tid * VW) = zt;
            }
            named_sync(1, NU);
            if (tid == 0) {
                __threadfence_block();
                s_zready = (int)(lk + 1);  // sz, sprow of this pass ready for the selection
                // this pass writes the previous pass's source, and CTA 0 the
                // basis entries of this pass's pivots: wait until every CTA's
                // selections so far are done reading both (as in the primal
                // kernel)
                const int ok = (int)wait_ctr(scnt, (unsigned)G * (lk + 1u), d->err, spin_limit);
                if (ok && g == 0) {
                    for (int k = 0; k < np; ++k) {
                        if (iters + k < d->trace_cap) {
                            d->trace[2 * (iters + k)] = pp[k];
                            d->trace[2 * (iters + k) + 1] = qq[k];
                        }
                        basis[pp[k]] = qq[k];
                    }
                    d->last_p = pp[np - 1];
                    d->last_q = qq[np - 1];
                }
                s_uok = ok;
            }
            named_sync(1, NU);
            const bool upd = active && s_uok;
            if (s_uok && tid < vpr) *reinterpret_cast<V *>(Bn + (long long)m * P + c0 + tid * VW) = zt;
            // Step 5 for the pass's pivots on the constraint rows of the strip
            if (upd && np == 2) {
                const V pr0 = *reinterpret_cast<const V *>(sprow[0] + lv * VW);
                const V pr1 = *reinterpret_cast<const V *>(sprow[1] + lv * VW);
                const int p0 = pp[0], p1 = pp[1];
                const T *__restrict__ c0p = pc[0];
                const T *__restrict__ c1p = pc[1];
                const T *abase = A + col0;
                T *bbase = Bn + col0;
                int i = lr;
                for (; i + 3 * rpp < m; i += 4 * rpp) {
                    const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                    V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    V t1 = ldv(reinterpret_cast<const V *>(abase + (long long)i1 * P));
                    V t2 = ldv(reinterpret_cast<const V *>(abase + (long long)i2 * P));
                    V t3 = ldv(reinterpret_cast<const V *>(abase + (long long)i3 * P));
                    t0 = pivot_vec<T>(t0, i, p0, c0p[i], pr0);
                    t1 = pivot_vec<T>(t1, i1, p0, c0p[i1], pr0);
                    t2 = pivot_vec<T>(t2, i2, p0, c0p[i2], pr0);
                    t3 = pivot_vec<T>(t3, i3, p0, c0p[i3], pr0);
                    *reinterpret_cast<V *>(bbase + (long long)i * P) = pivot_vec<T>(t0, i, p1, c1p[i], pr1);
                    *reinterpret_cast<V *>(bbase + (long long)i1 * P) = pivot_vec<T>(t1, i1, p1, c1p[i1], pr1);
                    *reinterpret_cast<V *>(bbase + (long long)i2 * P) = pivot_vec<T>(t2, i2, p1, c1p[i2], pr1);
                    *reinterpret_cast<V *>(bbase + (long long)i3 * P) = pivot_vec<T>(t3, i3, p1, c1p[i3], pr1);
                }
                for (; i < m; i += rpp) {
                    V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    t0 = pivot_vec<T>(t0, i, p0, c0p[i], pr0);
                    *reinterpret_cast<V *>(bbase + (long long)i * P) = pivot_vec<T>(t0, i, p1, c1p[i], pr1);
                }
            } else if (upd) {
                const V pr0 = *reinterpret_cast<const V *>(sprow[0] + lv * VW);
                const int p0 = pp[0];
                const T *__restrict__ c0p = pc[0];
                const T *abase = A + col0;
                T *bbase = Bn + col0;
                int i = lr;
                for (; i + 3 * rpp < m; i += 4 * rpp) {
                    const int i1 = i + rpp, i2 = i + 2 * rpp, i3 = i + 3 * rpp;
                    const V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    const V t1 = ldv(reinterpret_cast<const V *>(abase + (long long)i1 * P));
                    const V t2 = ldv(reinterpret_cast<const V *>(abase + (long long)i2 * P));
                    const V t3 = ldv(reinterpret_cast<const V *>(abase + (long long)i3 * P));
                    *reinterpret_cast<V *>(bbase + (long long)i * P) = pivot_vec<T>(t0, i, p0, c0p[i], pr0);
                    *reinterpret_cast<V *>(bbase + (long long)i1 * P) = pivot_vec<T>(t1, i1, p0, c0p[i1], pr0);
                    *reinterpret_cast<V *>(bbase + (long long)i2 * P) = pivot_vec<T>(t2, i2, p0, c0p[i2], pr0);
                    *reinterpret_cast<V *>(bbase + (long long)i3 * P) = pivot_vec<T>(t3, i3, p0, c0p[i3], pr0);
                }
                for (; i < m; i += rpp) {
                    const V t0 = ldv(reinterpret_cast<const V *>(abase + (long long)i * P));
                    *reinterpret_cast<V *>(bbase + (long long)i * P) = pivot_vec<T>(t0, i, p0, c0p[i], pr0);
                }
            }
        } else {
            // selection of the next pass's pivots a and b (dual simplex)
            int st = ST_RUNNING, nnp = 0, npend = ST_RUNNING;
            int pa = -1, qa = -1, pb = -1, qb = -1, rza = 0, rzb = 0;
            // The basic variable of row i after the pass.  CTA 0 writes the
            // basis entries of a pass's pivots during that pass, and this
            // selection runs before any wait of its own pass, so the entries
            // of the previous pass's pivots may not be in memory yet: they
            // are taken from ppv / qqv.  Older entries are: this CTA waited
            // in the previous pass for CTA 0's records, which CTA 0 publishes
            // only after finishing the pass before it.
            auto bkey = [&](int i) -> int {
                if (np > 1 && i == pp[1]) return qq[1];
                if (i == pp[0]) return qq[0];
                if (npv > 1 && i == ppv[1]) return qqv[1];
                if (i == ppv[0]) return qqv[0];
                return __ldcg(basis + i);
            };
            T *colA = nc[0];
            if (!select) {
                st = pend;  // the previous pass's selection already ended the solve
            } else {
                // the pass's pivot-row values at the rhs (the update warps' Step 4
                // values), from this CTA's copy of the source's rhs column: the
                // tableau's own rhs column belongs to one CTA, which may still be
                // writing it in the previous pass (no grid barrier separates the
                // passes)
                T pvr[kBlk];
                {
                    const T r = srhs[pp[0]] / pc[0][pp[0]];
                    pvr[0] = r;
                    pvr[1] = (T)0;
                    if (np > 1) {
                        const T t = (pp[1] == pp[0]) ? r : tfma(-pc[0][pp[1]], r, srhs[pp[1]]);
                        pvr[1] = t / pc[1][pp[1]];
                    }
                }
                named_sync(2, kSelThreads);  // every thread has read srhs[pp[.]] before it changes
                // ---- pivot a: the leaving row from the rhs of T2, every row
                // (from the rhs of T0 kept in scratch, which becomes T2's) ----
                Cand c = cand_empty();
                for (int i = stid; i < m; i += kSelThreads) {
                    const T h = blk_apply<T>(srhs[i], i, np, pp, pc, pvr);
                    srhs[i] = h;
                    const unsigned long long vk = okey(h);
                    if (vk < lim_r) cand_take(c, nbland ? zero_k : vk, nbland ? bkey(i) : i, i);
                }
                c = sel_min<SW>(c, 0ull, selc, selq, nullptr);
                if (c.idx < 0) st = ST_OPTIMAL;
                else if (iters + np >= iter_limit) st = ST_ITER_LIMIT;
                else if (c.idx >= m) st = ST_TIMEOUT;  // never: a row outside the tableau
                else pa = c.idx;
                if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                if (st == ST_RUNNING) {
                    // this pass's sprow and sz from the update warps
                    if (stid == 0) {
                        const long long t0 = clock64();
                        int ok = 1;
                        while (s_zready < (int)(lk + 1)) {
                            if (clock64() - t0 > spin_limit || *(volatile int *)d->err) {
                                atomicExch(d->err, 1);
                                ok = 0;
                                break;
                            }
                        }
                        s_sok = ok;
                    }
                    named_sync(2, kSelThreads);
                    __threadfence_block();
                    if (!s_sok) st = ST_TIMEOUT;
                }
                unsigned long long ka = 0ull;
                if (st == ST_RUNNING) {
                    // row r_a of T2 on this strip and its dual ratio test; the record
                    Cand e = cand_empty();
                    for (int j = c0 + stid; j < c1; j += kSelThreads) {
                        T x = lds(A + (long long)pa * P + j);
#pragma unroll
                        for (int k = 0; k < kBlk; ++k)
                            if (k < np)
                                x = (pa == pp[k]) ? sprow[k][j - c0] : tfma(-pc[k][pa], sprow[k][j - c0], x);
                        sra[j - c0] = x;
                        if (j < jend && okey(x) < lim_np)
                            cand_take(e, okey(pos_part(sz[j - c0]) / neg(x)), j, j);
                    }
                    e = sel_min<SW>(e, 0ull, selc, selq, nullptr);
                    if (stid == 0) {
                        recA[g] = e;
                        unsigned long long *v = valA + (size_t)g * kBlkVals;
                        for (int k = 0; k < np; ++k) v[k] = e.idx >= 0 ? tbits(sprow[k][e.idx - c0]) : 0ull;
                        red_add_release(rcnt, 1u);
                        s_sok = (int)wait_ctr(rcnt, tA, d->err, spin_limit);
                    }
                    named_sync(2, kSelThreads);
                    if (!s_sok) {
                        st = ST_TIMEOUT;
                    } else {
                        const Cand f = scan_records_tab<kSelThreads, kBlk>(recA, valA, G, stid, &ka, s_tab);
                        const Cand sel = sel_min<SW>(f, ka, selc, selq, &ka);
                        if (sel.idx < 0) st = ST_INFEASIBLE;
                        else if (sel.idx >= N - 1) st = ST_TIMEOUT;  // never
                        else {
                            qa = sel.idx;
                            rza = sel.vk == zero_k;
                        }
                        if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                    }
                }
                if (st == ST_RUNNING) {
                    // column q_a of T2, every row: the next pass's first pivot column
                    T pvq[kBlk];
#pragma unroll
                    for (int k = 0; k < kBlk; ++k) pvq[k] = tfrom<T>(s_tab[ka * kBlk + k]);
                    // the objective row's entry rides with the first batch
                    const T am = stid == 0 ? lds(A + (long long)m * P + qa) : (T)0;
                    for (int i0 = stid; i0 < m; i0 += kColRows * kSelThreads) {
                        T av[kColRows];
#pragma unroll
                        for (int u = 0; u < kColRows; ++u) {
                            const int i = i0 + u * kSelThreads;
                            av[u] = i < m ? lds(A + (long long)i * P + qa) : (T)0;
                        }
#pragma unroll
                        for (int u = 0; u < kColRows; ++u) {
                            const int i = i0 + u * kSelThreads;
                            if (i >= m) break;
                            colA[i] = blk_apply<T>(av[u], i, np, pp, pc, pvq);
                        }
                    }
                    if (stid == 0) colA[m] = blk_apply<T>(am, m, np, pp, pc, pvq);
                    named_sync(2, kSelThreads);
                    // ---- pivot b: the rhs after pivot a and its leaving row ----
                    const T piva = colA[pa];
                    const T pra = srhs[pa] / piva;  // pivot a's row at the rhs
                    const int nblandb = (rza ? deg + 1 : 0) >= bland_after;
                    Cand cb2 = cand_empty();
                    for (int i = stid; i < m; i += kSelThreads) {
                        const T h = (i == pa) ? pra : tfma(-colA[i], pra, srhs[i]);
                        const unsigned long long vk = okey(h);
                        if (vk < lim_r)
                            cand_take(cb2, nblandb ? zero_k : vk,
                                      nblandb ? (i == pa ? qa : bkey(i)) : i, i);
                    }
                    cb2 = sel_min<SW>(cb2, 0ull, selc, selq, nullptr);
                    nnp = 1;
                    if (cb2.idx < 0) npend = ST_OPTIMAL;
                    else if (iters + np + 1 >= iter_limit) npend = ST_ITER_LIMIT;
                    else if (cb2.idx >= m) st = ST_TIMEOUT;  // never
                    else pb = cb2.idx;
                    if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                    if (st == ST_RUNNING && pb >= 0) {
                        // row r_b after pivot a on this strip, its dual ratio test;
                        // the record carries the pivot-row values at its column
                        Cand e = cand_empty();
                        const T cab = colA[pb], cam = colA[m];
                        for (int j = c0 + stid; j < c1; j += kSelThreads) {
                            T x = lds(A + (long long)pb * P + j);
#pragma unroll
                            for (int k = 0; k < kBlk; ++k)
                                if (k < np)
                                    x = (pb == pp[k]) ? sprow[k][j - c0] : tfma(-pc[k][pb], sprow[k][j - c0], x);
                            const T prj = sra[j - c0] / piva;  // pivot a's row at column j
                            x = (pb == pa) ? prj : tfma(-cab, prj, x);
                            if (j < jend && okey(x) < lim_np) {
                                const T z3 = tfma(-cam, prj, sz[j - c0]);
                                cand_take(e, okey(pos_part(z3) / neg(x)), j, j);
                            }
                        }
                        e = sel_min<SW>(e, 0ull, selc, selq, nullptr);
                        if (stid == 0) {
                            recB[g] = e;
                            unsigned long long *v = valB + (size_t)g * kBlkVals;
                            for (int k = 0; k < np; ++k) v[k] = e.idx >= 0 ? tbits(sprow[k][e.idx - c0]) : 0ull;
                            v[np] = e.idx >= 0 ? tbits(sra[e.idx - c0] / piva) : 0ull;
                            red_add_release(rcnt, 1u);
                            s_sok = (int)wait_ctr(rcnt, tB, d->err, spin_limit);
                        }
                        named_sync(2, kSelThreads);
                        unsigned long long kb = 0ull;
                        if (!s_sok) {
                            st = ST_TIMEOUT;
                        } else {
                            const Cand f = scan_records_tab<kSelThreads, kBlk + 1>(recB, valB, G, stid, &kb, s_tab);
                            const Cand sel = sel_min<SW>(f, kb, selc, selq, &kb);
                            if (sel.idx < 0) npend = ST_INFEASIBLE;
                            else if (sel.idx >= N - 1) st = ST_TIMEOUT;  // never
                            else {
                                qb = sel.idx;
                                rzb = sel.vk == zero_k;
                            }
                            if (st == ST_TIMEOUT && stid == 0) atomicExch(d->err, 1);
                        }
                        if (st == ST_RUNNING && qb >= 0) {
                            // column q_b after pivot a, every row
                            T pvb[kBlk + 1];
#pragma unroll
                            for (int k = 0; k <= kBlk; ++k) pvb[k] = tfrom<T>(s_tab[kb * (kBlk + 1) + k]);
                            T *colB = nc[1];
                            const T am = stid == 0 ? lds(A + (long long)m * P + qb) : (T)0;
                            for (int i0 = stid; i0 < m; i0 += kColRows * kSelThreads) {
                                T av[kColRows];
#pragma unroll
                                for (int u = 0; u < kColRows; ++u) {
                                    const int i = i0 + u * kSelThreads;
                                    av[u] = i < m ? lds(A + (long long)i * P + qb) : (T)0;
                                }
#pragma unroll
                                for (int u = 0; u < kColRows; ++u) {
                                    const int i = i0 + u * kSelThreads;
                                    if (i >= m) break;
                                    const T t = blk_apply<T>(av[u], i, np, pp, pc, pvb);
                                    colB[i] = (i == pa) ? pvb[np] : tfma(-colA[i], pvb[np], t);
                                }
                            }
                            if (stid == 0)  // pa < m
                                colB[m] = tfma(-colA[m], pvb[np], blk_apply<T>(am, m, np, pp, pc, pvb));
                            nnp = 2;
                        }
                    }
                }
            }
            // every selection thread is done reading this pass's source
            named_sync(2, kSelThreads);
            if (stid == 0) {
                if (st != ST_TIMEOUT) red_add_release(scnt, 1u);
                s_status = st;
                s_np = nnp;
                s_pend = npend;
                s_p[0] = pa;
                s_q[0] = qa;
                s_p[1] = pb;
                s_q[1] = qb;
                s_rz[0] = rza;
                s_rz[1] = rzb;
            }
        }
        // the CTA's pass and its selection of the next pass are done
        if (tid == 0) {
            s_abort = ab;  // past the host's deadline: stop, and end every CTA's waits
            if (ab) atomicExch(d->err, 1);
        }
        __syncthreads();
        iters += np;
        ++lk;
        status = s_abort ? ST_TIMEOUT : s_status;
        if (!s_uok) status = ST_TIMEOUT;
        if (status == ST_RUNNING) {
            npv = np;
            np = s_np;
            pend = s_pend;
            for (int k = 0; k < kBlk; ++k) {
                ppv[k] = pp[k];
                qqv[k] = qq[k];
                pp[k] = s_p[k];
                qq[k] = s_q[k];
            }
            deg = s_rz[0] ? deg + 1 : 0;
            if (np > 1) deg = s_rz[1] ? deg + 1 : 0;
            cb = (cb + 2) & 3;
        }
        cur ^= 1;
        // no grid barrier between passes (as in the primal kernel)
    }

    if (g == 0 && tid == 0) {
        // every CTA's last selection is done, and with it its last wait
        wait_ctr(scnt, (unsigned)G * (lk + 1u), d->err, spin_limit);
        d->status = (*(volatile int *)d->err) ? ST_TIMEOUT : status;
        d->iters = iters;
        d->iter_limit = iter_limit;
        d->deg = deg;
        d->T = bufs[cur];  // hand over the buffer holding the last tableau
        d->T2 = bufs[cur ^ 1];
    }
}

}  // namespace

// CTAs of up to this many threads launch the FP64 two-pivot primal kernel
// compiled for it: up to 80 registers a thread instead of 64, so the
// selection chain and the update keep their values in registers (the
// 1024-thread build spills)
constexpr int kMidThreads = 768;
// and of up to this many: 96 registers
constexpr int kSmallThreads = 640;

cudaError_t launch_pivot_pipe(int prec, LpDesc *d_desc, const PivotShape &sh,
                              long long spin_limit, long long budget, cudaStream_t s) {
    int W = sh.strip;
    int dbm = sh.pipe == 2 ? 1 : 0;
    void *args[] = {&d_desc, &W, &spin_limit, &budget, &dbm};
    if (sh.pipe == 3) {  // two pivots per pass
        int split = sh.split;
        void *bargs[] = {&d_desc, &W, &spin_limit, &budget};
        void *pargs[] = {&d_desc, &W, &split, &spin_limit, &budget};
        const bool w8 = sh.sel_warps == 8;
        const void *fn = sh.dual ? (prec == PREC_FP64
                                        ? (w8 ? (const void *)pivot_block_dual_kernel<double, 8>
                                              : (const void *)pivot_block_dual_kernel<double, 4>)
                                        : (w8 ? (const void *)pivot_block_dual_kernel<float, 8>
                                              : (const void *)pivot_block_dual_kernel<float, 4>))
                         : prec == PREC_FP64
                             ? (sh.split > 0
                                    ? (w8 ? (sh.dist ? (const void *)pivot_block_kernel<double, 8, true, true>
                                                     : (const void *)pivot_block_kernel<double, 8, false, true>)
                                          : (sh.dist ? (const void *)pivot_block_kernel<double, 4, true, true>
                                                     : (const void *)pivot_block_kernel<double, 4, false, true>))
                                    : (w8 ? (sh.threads <= kSmallThreads
                                                 ? (sh.dist ? (const void *)pivot_block_kernel<double, 8, true, false, kSmallThreads>
                                                            : (const void *)pivot_block_kernel<double, 8, false, false, kSmallThreads>)
                                             : sh.threads <= kMidThreads
                                                 ? (sh.dist ? (const void *)pivot_block_kernel<double, 8, true, false, kMidThreads>
                                                            : (const void *)pivot_block_kernel<double, 8, false, false, kMidThreads>)
                                                 : (sh.dist ? (const void *)pivot_block_kernel<double, 8, true, false>
                                                            : (const void *)pivot_block_kernel<double, 8, false, false>))
                                          : (sh.dist ? (const void *)pivot_block_kernel<double, 4, true, false>
                                                     : (const void *)pivot_block_kernel<double, 4, false, false>)))
                             : (sh.split > 0
                                    ? (w8 ? (sh.dist ? (const void *)pivot_block_kernel<float, 8, true, true>
                                                     : (const void *)pivot_block_kernel<float, 8, false, true>)
                                          : (sh.dist ? (const void *)pivot_block_kernel<float, 4, true, true>
                                                     : (const void *)pivot_block_kernel<float, 4, false, true>))
                                    : (w8 ? (sh.dist ? (const void *)pivot_block_kernel<float, 8, true, false>
                                                     : (const void *)pivot_block_kernel<float, 8, false, false>)
                                          : (sh.dist ? (const void *)pivot_block_kernel<float, 4, true, false>
                                                     : (const void *)pivot_block_kernel<float, 4, false, false>)));
        if (sh.smem_bytes > 0) {  // static shared memory counts against the 48 KB default too
            cudaError_t e = allow_dyn_smem(fn);
            if (e != cudaSuccess) return e;
        }
        return cudaLaunchCooperativeKernel(fn, dim3(sh.ctas), dim3(sh.threads),
                                           sh.dual ? bargs : pargs, sh.smem_bytes, s);
    }
    if (sh.dual) {
        const void *fn = prec == PREC_FP64 ? (const void *)pivot_pipe_dual_kernel<double, 4>
                                           : (const void *)pivot_pipe_dual_kernel<float, 4>;
        if (sh.smem_bytes > 0) {  // static shared memory counts against the 48 KB default too
            cudaError_t e = allow_dyn_smem(fn);
            if (e != cudaSuccess) return e;
        }
        return cudaLaunchCooperativeKernel(fn, dim3(sh.ctas), dim3(sh.threads), args,
                                           sh.smem_bytes, s);
    }
    const void *fn = prec == PREC_FP64
                         ? (sh.pipe == 2 ? (const void *)pivot_pipe_kernel<double, 2>
                                         : (const void *)pivot_pipe_kernel<double, 4>)
                         : (sh.pipe == 2 ? (const void *)pivot_pipe_kernel<float, 2>
                                         : (const void *)pivot_pipe_kernel<float, 4>);
    if (sh.smem_bytes > 0) {  // static shared memory counts against the 48 KB default too
        cudaError_t e = allow_dyn_smem(fn);
        if (e != cudaSuccess) return e;
    }
    return cudaLaunchCooperativeKernel(fn, dim3(sh.ctas), dim3(sh.threads), args, sh.smem_bytes, s);
}

// Launch shape of the pipelined kernel: strips sized for the update threads
// (all but the last warp), shared memory for the strip and the selection
// warp's block of rows.
PivotShape choose_pipe_shape(int prec, int M, long long P, int sms, int threads, int ctas,
                             int dual, int split) {
    PivotShape sh;
    const int vw = prec == PREC_FP64 ? 2 : 4, sector = prec == PREC_FP64 ? 4 : 8;
    const size_t esz = prec == PREC_FP64 ? sizeof(double) : sizeof(float);
    // Default CTA size.  The one-pivot kernels take 1024 threads.  The
    // two-pivot kernels size their update threads so that each forms about
    // 25 + m / 68 rows of its vector column per pass: where the selection
    // chain bounds the pass, fewer update threads leave it more of the memory
    // system, and a longer chain (more rows) hides a longer update.  Measured
    // pivot-kernel us per pivot at 512 / 640 / 768 / 1024 threads (rule's
    // choice marked *): 512 x 4096 11.3* / 11.6 / 12.1 / 12.2, 256 x 8192
    // 10.6* / 11.0 / 11.2 / 11.5, 1024^2 13.3* / 13.2 / 13.7 / 14.1, 1536^2
    // 17.6 / 16.9* / 17.9 / 19.4, 1024 x 4096 19.5 / 17.0 / 17.2* (704) /
    // 18.8, 2048^2 35.6 / 26.3 / 23.0* / 24.5 (dual form 35.1 / 28.3 / 25.7* /
    // 27.2), 3072^2 73.1 / 53.5 / 45.3 / 42.5*, 4096 x 512 70.0 / 52.6 / 43.8
    // / 41.0*, 8192^2 201 / 160 / 150 / 147*.  With vectors
    // left in place only the structural share of the columns counts.
    if (threads > 0) {
        sh.threads = threads;
    } else if (dual >= 2) {
        const long long g0 = (long long)M * P >= (1ll << 19) ? sms : (sms + 1) / 2;
        long long w0 = (P + g0 - 1) / g0;
        w0 = (w0 + sector - 1) / sector * sector;
        double vpr = (double)w0 / vw;
        if (split > 0) vpr *= (double)split / (double)P;
        const int m = M - 1;
        const double rows = 25.0 + m / 68.0;
        const int sel = (long long)M * P * (long long)esz < (384ll << 20) ? 256 : 128;
        const double nu_want = m * vpr / rows;
        sh.threads = (int)((nu_want + sel) / 32.0 + 0.5) * 32;
    } else {
        sh.threads = kMaxThreads;
    }
    sh.threads = std::min(kMaxThreads, std::max(2 * kSelThreadsMax, (sh.threads + 31) / 32 * 32));
    const int nu = sh.threads - kSelThreadsMax;
    // Default grid: every SM.  A pivot costs the selection chain plus the
    // update of one strip, and a narrower strip shortens the update while the
    // extra pricing records add little (512 x 4096: 11.7 us per pivot on 152
    // CTAs, 14.5 on 73).  Below half a million tableau elements the records
    // weigh more than the update saved, and half the SMs does as well.
    const long long g_auto = (long long)M * P >= (1ll << 19) ? sms : (sms + 1) / 2;
    long long g = ctas > 0 ? ctas : g_auto;
    const long long gmin = (P + (long long)nu * vw - 1) / ((long long)nu * vw);
    g = std::max<long long>(std::max<long long>(g, gmin), 1);
    long long w = (P + g - 1) / g;
    w = (w + sector - 1) / sector * sector;
    if (w > (long long)nu * vw) w = (long long)nu * vw / sector * sector;
    sh.strip = (int)w;
    sh.ctas = (int)((P + w - 1) / w);
    // two runs per CTA (the two-pivot primal kernel): the widest CTA sizes
    // the shared memory; every CTA needs columns and at most a pass of the
    // update threads
    if (dual == 2 && split > 0 && split % sector == 0 && split < P) {
        int wmax = 0;
        bool fits = true;
        for (int k = 0; k < sh.ctas && fits; ++k) {
            const Strip st = make_strip(k, sh.ctas, sh.strip, split, P, sector);
            fits = st.w() > 0 && st.w() <= nu * vw;
            wmax = std::max(wmax, st.w());
        }
        if (fits) {
            // (two sectors more: the kernel may deal the slack vectors out
            // by load, one CTA getting up to a few vectors above its run)
            sh.split = split;
            sh.strip = std::max(wmax, std::min(wmax + 2 * sector, nu * vw / sector * sector));
            w = sh.strip;
        }
    }
    // the pivot columns of two pivots and the ratio numerators and screening
    // keys (primal), or the strip of the new objective row (dual)
    const size_t cbytes = ((size_t)M * esz + 15) & ~(size_t)15;
    const size_t sprow = ((size_t)w * esz + 15) & ~(size_t)15;
    // (dual == 2: the two-pivot kernel, four pivot rows and columns)
    // (dual == 3: the two-pivot dual kernel, four pivot rows and columns and the rhs)
    const size_t scratch = dual == 1   ? sprow + 2 * cbytes
                           : dual == 2 ? 5 * cbytes + (size_t)M * sizeof(unsigned long long)
                           : dual == 3 ? 5 * cbytes
                                       : 3 * cbytes + (size_t)M * sizeof(unsigned long long);
    const size_t fixed = dual >= 2 ? 4 * sprow : sprow;
    if (fixed + scratch <= kMaxDynSmem) {
        sh.use_smem = 1;
        sh.smem_bytes = fixed + scratch;
        sh.scratch_stride = 0;
    } else {
        sh.use_smem = 0;
        sh.smem_bytes = fixed;
        sh.scratch_stride = (long long)((scratch + 255) & ~(size_t)255);
    }
    sh.dual = dual == 1 || dual == 3;
    // one CTA per SM at 1024 threads: the grid must fit the SMs (cooperative
    // launch), the strip one pass of the update threads
    sh.pipe = sh.ctas <= sms && (long long)sh.strip <= (long long)nu * vw &&
              (dual < 2 || sh.ctas <= kMaxRecs);
    return sh;
}

}  // namespace gbs
