// C ABI of the tableau simplex library (declared in include/gbsimplex.h).
//
// A handle owns, on its device: the input copies (A, b, c in FP64), the
// pitched tableau, the basis, the staged pivot column, the per-CTA partials,
// the barrier words, the pivot trace and a small descriptor/state block.  All
// of it is allocated on lp_load (reused when the next LP fits) and freed on
// lp_destroy.

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stddef.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <new>
#include <thread>

#include "gbs_internal.h"
#include "gbsimplex.h"

using namespace gbs;

// From this many tableau elements on, the primal simplex applies two pivots
// per pass (double-buffered, half the tableau traffic per pivot); below it
// the pipelined kernel runs in place, whose shorter chain wins on small
// tableaus.  Measured per pivot, FP64, one pivot per pass in place / two per
// pass: 256^2 9.3 / 9.4 us, 512^2 10.4 / 10.3, 1024^2 14.2 / 13.3, 2048^2
// 27.5 / 24.3, 3000^2 65.6 / 41.4 (the in-place tableau no longer fits L2).
constexpr long long kBlockElems = 1ll << 19;
// Below this size the two-pivot selection is the longer chain and gets eight
// warps, from it on four (measured: 4096 x 512 (152 MB) 51.3 us per pivot
// with eight, 60.5 with four, 57.9 with one pivot per pass; 8192^2 FP64
// (1.07 GB) 249 with four, 253 with eight, 370 with one pivot per pass).
constexpr size_t kBlockBytes = 384ull << 20;
// The two-pivot primal kernel distributes its ratio test over the CTAs (one
// more record exchange per pivot, a slice of the column's rows per CTA) when
// every selection thread would otherwise form more than this many rows of
// each new column (measured per pivot, redundant / distributed: 512 x 4096
// (2 rows a thread) 11.4 / 13.5 us, 2048^2 (8) 24.3 / 23.7, 4096 x 512 (16)
// 46.6 / 40.5, 8192^2 (64) 243 / 239).
constexpr int kDistRows = 4;
// smallest tableau (elements) on which the two-pivot primal kernel leaves
// vectors in place (lp_options.zero_skip)
constexpr long long kSkipElems = 1ll << 25;

struct lp_handle {
    lp_options opt;
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char err[512] = {0};

    // problem
    bool loaded = false;
    bool solved = false;
    int m = 0, n = 0, M = 0, N = 0, sense = 0, prec = PREC_FP64;
    int phase = 0;  // Phase I (primal form, some b_i < 0): 1 in Phase 1, 2 after it; 0 without
    long long P = 0;
    double eps_d = 0, eps_p = 0, eps_r = 0;

    // device memory
    double *dA = nullptr, *db = nullptr, *dc = nullptr;
    size_t cap_A = 0, cap_b = 0, cap_c = 0;  // element capacities
    void *dT = nullptr;                         // the current tableau
    size_t cap_T = 0;                           // bytes
    void *dT2 = nullptr;                        // double-buffered pipelined kernel
    size_t cap_T2 = 0;
    void *dcolx = nullptr;                      // two-pivot kernel: four pivot-column slots
    size_t cap_colx = 0;
    int *dbasis = nullptr;
    size_t cap_basis = 0;
    void *dscratch = nullptr;
    size_t cap_scratch = 0;                     // bytes
    Cand *dpart = nullptr;                      // 38 * max_ctas (records, values)
    int max_ctas = 0;
    unsigned *dbar = nullptr;                   // kBarWords: barrier, counters, err
    int *dtrace = nullptr;
    long long cap_trace = 0;
    LpDesc *ddesc = nullptr;
    InputStats *dstats = nullptr;
    double *dx = nullptr, *dy = nullptr, *dobj = nullptr;
    size_t cap_x = 0, cap_y = 0;
    // a caller's device range that the buffers above (from dA to dy, not the
    // descriptor, statistics, barrier and objective words) and the FP64
    // reinversion buffers below are carved from instead of cudaMalloc:
    // bump-allocated, never freed (handle_bind_region)
    unsigned char *region = nullptr;
    size_t region_size = 0, region_used = 0;

    // descriptor as written by lp_load, and a pinned mirror of the device copy
    // read back after each solve
    LpDesc desc{};
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the pivot kernel
    LpDesc *pdesc = nullptr;
    double *pobj = nullptr;
    PivotShape shape{};
    PivotShape shape_alt{};  // the other pivot rule (FP32 recovery), same strips

    // FP32 mode: FP64 reinversion buffers and per-solve accounting
    ReinvBufs rb{};
    size_t cap_W = 0;       // doubles in rb.W
    size_t cap_rb = 0;      // rows the index/vector buffers hold
    double fp32_kernel_ms = 0.0, reinv_ms = 0.0;
    int fp32_launches = 0, reinversions = 0;
    double eps32_d = 0, eps32_p = 0, eps32_r = 0;

    // wall-clock limit (opt.time_limit_s): the abort word the pivot kernels
    // poll, in mapped pinned host memory, and the deadline of the solve in
    // flight
    int *habort = nullptr;        // host view
    int *dabort = nullptr;        // device view of the same word
    std::chrono::steady_clock::time_point deadline{};
    bool timed_out = false;       // the last solve ended in LP_TIMEOUT: reload first

    // FP32 mode: emulated-FP64 products of the body refresh, and its time
    OzWork oz{};
    double body_ms = 0.0;
    int last_ns = 0;  // structural basics of the last reinversion
};

namespace {

thread_local char g_err[512];

void set_err(lp_handle *h, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(h ? h->err : g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

#define CUDA_TRY(h, call)                                                           \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) {                                                    \
            set_err((h), "%s failed: %s", #call, cudaGetErrorString(e_));           \
            return e_ == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA;      \
        }                                                                           \
    } while (0)

// A device buffer from cudaMalloc, or on a handle bound to a device range,
// the next 256-byte-aligned piece of that range.
cudaError_t dev_alloc(lp_handle *h, void **ptr, size_t bytes) {
    if (!h->region) return cudaMalloc(ptr, bytes);
    const size_t at = (h->region_used + 255) & ~(size_t)255;
    if (at > h->region_size || bytes > h->region_size - at) return cudaErrorMemoryAllocation;
    *ptr = h->region + at;
    h->region_used = at + bytes;
    return cudaSuccess;
}

void dev_free(lp_handle *h, void *p) {
    if (p && !h->region) cudaFree(p);
}

template <typename P>
cudaError_t grow(lp_handle *h, P **ptr, size_t *cap, size_t need_elems) {
    if (*ptr && *cap >= need_elems) return cudaSuccess;
    dev_free(h, *ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = dev_alloc(h, (void **)ptr, std::max<size_t>(need_elems, 1) * sizeof(P));
    if (e == cudaSuccess) *cap = need_elems;
    return e;
}

cudaError_t grow_bytes(lp_handle *h, void **ptr, size_t *cap, size_t bytes) {
    if (*ptr && *cap >= bytes) return cudaSuccess;
    dev_free(h, *ptr);
    *ptr = nullptr;
    *cap = 0;
    cudaError_t e = dev_alloc(h, ptr, std::max<size_t>(bytes, 16));
    if (e == cudaSuccess) *cap = bytes;
    return e;
}

double bits_to_double(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

}  // namespace

void gbs::set_last_error_global(const char *msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
}

extern "C" {

void lp_options_default(lp_options *o) {
    if (!o) return;
    memset(o, 0, sizeof *o);
    o->precision = LP_FP64;
    o->reinv_k = 50;
    o->max_iters = 1000000000000ll;
    o->eps_d = 0.0;
    o->eps_p = 0.0;
    o->eps_r = 0.0;
    o->bland_after = 32;
    o->threads = 0;
    o->spin_timeout_cycles = 4000000000ll;
    o->cuda_stream = nullptr;
    o->device = 0;
    o->ctas = 0;
    o->trace_cap = 0;
    o->group_elems = 0;
    o->pipeline = 1;
    o->reinv_body = 1;
    o->zero_skip = 1;
    o->spill_pivots = 0;
    o->lanes = 3;
}

const char *lp_version(void) { return "gbsimplex 0.1 (sm_103a)"; }

size_t lp_options_size(void) { return sizeof(lp_options); }

const char *lp_last_error(const lp_handle *h) { return h ? h->err : g_err; }

lp_err lp_create(lp_handle **out, const lp_options *opt) {
    if (!out) {
        set_err(nullptr, "lp_create: out is NULL");
        return LP_ERR_INVALID_ARG;
    }
    *out = nullptr;
    lp_options o;
    if (opt) o = *opt; else lp_options_default(&o);
    if (o.precision != LP_FP64 && o.precision != LP_FP32_REINV) {
        set_err(nullptr, "lp_create: unknown precision %d", o.precision);
        return LP_ERR_INVALID_ARG;
    }
    if (o.max_iters < 0 || o.bland_after < 0 || o.trace_cap < 0 || o.spin_timeout_cycles <= 0 ||
        o.threads < 0 || o.threads > 1024 || o.ctas < 0 || o.reinv_k < 1) {
        set_err(nullptr, "lp_create: option out of range");
        return LP_ERR_INVALID_ARG;
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev <= 0) {
        set_err(nullptr, "lp_create: no CUDA device (%s)", cudaGetErrorString(e));
        return LP_ERR_CUDA;
    }
    if (o.device < 0 || o.device >= ndev) {
        set_err(nullptr, "lp_create: device %d out of range (%d devices)", o.device, ndev);
        return LP_ERR_INVALID_ARG;
    }
    lp_handle *h = new (std::nothrow) lp_handle();
    if (!h) {
        set_err(nullptr, "lp_create: host allocation failed");
        return LP_ERR_OOM;
    }
    h->opt = o;
    h->device = o.device;
    h->prec = o.precision == LP_FP64 ? PREC_FP64 : PREC_FP32;
    DeviceRestore restore_;
    e = cudaSetDevice(h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) {
        if (o.cuda_stream) {
            h->stream = (cudaStream_t)o.cuda_stream;
        } else {
            e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
            h->own_stream = e == cudaSuccess;
        }
    }
    if (e == cudaSuccess) e = cudaMalloc(&h->ddesc, sizeof(LpDesc));
    if (e == cudaSuccess) e = cudaMalloc(&h->dstats, sizeof(InputStats));
    // the synchronisation block, then the two-pivot kernels' update counts
    if (e == cudaSuccess) e = cudaMalloc(&h->dbar, (kBarWords + 4) * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&h->dobj, sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&h->pdesc, sizeof(LpDesc));
    if (e == cudaSuccess) e = cudaMallocHost(&h->pobj, sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&h->ev1);
    if (e == cudaSuccess) e = cudaHostAlloc(&h->habort, sizeof(int), cudaHostAllocMapped);
    if (e == cudaSuccess) {
        *h->habort = 0;
        e = cudaHostGetDevicePointer((void **)&h->dabort, h->habort, 0);
    }
    if (e != cudaSuccess) {
        set_err(nullptr, "lp_create: %s", cudaGetErrorString(e));
        lp_destroy(h);
        return e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA;
    }
    *out = h;
    return LP_OK;
}

void lp_destroy(lp_handle *h) {
    if (!h) return;
    DeviceRestore restore_;
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    void *rbufs[] = {h->rb.Lflag, h->rb.S, h->rb.R, h->rb.posS, h->rb.posR, h->rb.counts,
                     h->rb.pivrow, h->rb.W, h->rb.xS, h->rb.yR, h->rb.zrow, h->rb.rhs, h->rb.chk,
                     h->rb.bar};
    for (void *p : rbufs) dev_free(h, p);
    void *grown[] = {h->dA, h->db, h->dc, h->dT, h->dT2, h->dcolx, h->dbasis, h->dscratch,
                     h->dpart, h->dtrace, h->dx, h->dy};
    for (void *p : grown) dev_free(h, p);
    void *bufs[] = {h->dbar, h->ddesc, h->dstats, h->dobj};
    for (void *p : bufs)
        if (p) cudaFree(p);
    if (h->pdesc) cudaFreeHost(h->pdesc);
    if (h->pobj) cudaFreeHost(h->pobj);
    if (h->habort) cudaFreeHost(h->habort);
    oz_work_free(h->oz);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

lp_err lp_load(lp_handle *h, int m, int n, const double *A, const double *b, const double *c,
               lp_sense sense) {
    if (!h) return LP_ERR_INVALID_ARG;
    h->err[0] = 0;
    if (m < 1 || n < 1 || !A || !b || !c) {
        set_err(h, "lp_load: need m, n >= 1 and non-NULL A, b, c (m=%d n=%d)", m, n);
        return LP_ERR_INVALID_ARG;
    }
    if (sense != LP_MAX_LE && sense != LP_MIN_GE) {
        set_err(h, "lp_load: unknown sense %d", (int)sense);
        return LP_ERR_INVALID_ARG;
    }
    if ((long long)n + m + 1 > 0x7fffffffll - 64) {
        set_err(h, "lp_load: n + m too large");
        return LP_ERR_INVALID_ARG;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    h->loaded = false;
    h->solved = false;
    h->timed_out = false;
    const int M = m + 1, N = n + m + 1;
    const long long P = pitch_for(N);
    const size_t esz = h->prec == PREC_FP64 ? sizeof(double) : sizeof(float);
    // the inputs, and what they allow: a primal form with some b_i < 0 goes
    // through Phase I (FP64 single solves; not in the paper)
    CUDA_TRY(h, grow(h, &h->dA, &h->cap_A, (size_t)m * n));
    CUDA_TRY(h, grow(h, &h->db, &h->cap_b, (size_t)m));
    CUDA_TRY(h, grow(h, &h->dc, &h->cap_c, (size_t)n));
    InputStats st;
    {
        cudaStream_t s0 = h->stream;
        CUDA_TRY(h, cudaMemcpyAsync(h->dA, A, sizeof(double) * (size_t)m * n, cudaMemcpyDefault, s0));
        CUDA_TRY(h, cudaMemcpyAsync(h->db, b, sizeof(double) * (size_t)m, cudaMemcpyDefault, s0));
        CUDA_TRY(h, cudaMemcpyAsync(h->dc, c, sizeof(double) * (size_t)n, cudaMemcpyDefault, s0));
        CUDA_TRY(h, launch_inspect(h->dA, h->db, h->dc, m, n, h->dstats, s0));
        CUDA_TRY(h, cudaMemcpyAsync(&st, h->dstats, sizeof st, cudaMemcpyDeviceToHost, s0));
        CUDA_TRY(h, cudaStreamSynchronize(s0));
    }
    if (st.flags & 4) {
        set_err(h, "lp_load: A, b or c holds a NaN or infinity");
        return LP_ERR_INVALID_ARG;
    }
    const bool phase1 = sense == LP_MAX_LE && (st.flags & 1);
    if (phase1 && h->prec != PREC_FP64) {
        set_err(h, "lp_load: max form with some b < 0 needs Phase I, which the FP64 mode has "
                   "(the FP32 mode needs b >= 0)");
        return LP_ERR_INFEASIBLE_START;
    }
    if (sense == LP_MIN_GE && (st.flags & 2)) {
        set_err(h, "lp_load: min form needs c >= 0 (the slack basis must be dual feasible)");
        return LP_ERR_INFEASIBLE_START;
    }
    // the pipelined kernels where they can take the LP: the primal rule in
    // place for small tableaus and two pivots per pass above, the dual rule
    // double-buffered (the rule runs for its sense, and in FP32 mode for both)
    if (h->opt.pipeline < 0 || h->opt.pipeline > 5) {
        set_err(h, "lp_load: unknown pipeline mode %d", h->opt.pipeline);
        return LP_ERR_INVALID_ARG;
    }
    const bool primal = sense == LP_MAX_LE || h->prec == PREC_FP32;
    const bool dualr = sense == LP_MIN_GE || h->prec == PREC_FP32 || phase1;
    int pmode = primal ? h->opt.pipeline : 0;
    const bool force_dist = pmode == 5;  // 5: as 4, the ratio test always distributed
    if (pmode == 5) pmode = 4;
    const size_t tbytes = (size_t)M * P * esz;
    if (pmode == 1) pmode = (long long)M * P >= kBlockElems ? 4 : 2;
    const bool dwant = dualr && h->opt.pipeline != 0;
    bool have_t2 = false;
    if (pmode >= 3 || dwant) {
        have_t2 = grow_bytes(h, &h->dT2, &h->cap_T2, (size_t)M * P * esz) == cudaSuccess;
        if (!have_t2) cudaGetLastError();
    }
    if (pmode >= 3 && !have_t2) {
        if (h->opt.pipeline >= 3) {
            set_err(h, "lp_load: no device memory for the second tableau buffer (pipeline 3)");
            return LP_ERR_OOM;
        }
        pmode = 2;  // automatic mode without room for a second buffer: in place
    }
    if (pmode == 4)  // the two-pivot kernel's pivot-column slots
        CUDA_TRY(h, grow_bytes(h, &h->dcolx, &h->cap_colx, 4 * (((size_t)M * esz + 15) & ~(size_t)15)));
    const bool dpipe = dwant && have_t2;
    // the two-pivot primal kernel's second run of columns (with zero_skip):
    // the slack and rhs columns, from the last whole sector of
    // the structural columns.  Only where the update bounds the pass: on
    // tableaus of at least kSkipElems elements with at least one slack
    // column per four structural ones.  On the smaller tableaus the
    // selection chain bounds the pass and an update that finishes early only
    // crowds the chain's loads (4096 x 512 of the paper's family: 63 against
    // 42 us per pivot; 2048^2: 27 against 25).  zero_skip 2: at any size.
    const bool skip = h->opt.zero_skip == 2 ||
                      (h->opt.zero_skip == 1 && 4ll * m >= n && (long long)M * P >= kSkipElems);
    const int sector = h->prec == PREC_FP64 ? 4 : 8;
    const int split = skip ? n / sector * sector : 0;
    auto shape_for = [&](int rule) {
        if (rule == 0 && pmode) {
            PivotShape ps = choose_pipe_shape(h->prec, M, P, h->sms, h->opt.threads, h->opt.ctas,
                                              pmode == 4 ? 2 : 0, pmode == 4 ? split : 0);
            if (ps.pipe) {
                if (pmode == 3) ps.pipe = 2;  // double-buffered
                if (pmode == 4) {  // double-buffered, two pivots per pass
                    ps.pipe = 3;
                    ps.sel_warps = tbytes < kBlockBytes ? 8 : 4;
                    // each CTA forms the new columns on its own rows once the
                    // whole columns would take a selection thread more than
                    // kDistRows rows
                    ps.dist = force_dist || m > kDistRows * 32 * ps.sel_warps;
                }
                return ps;
            }
        }
        if (rule == 1 && dpipe) {
            // the dual rule: two pivots per pass unless one is asked for (2, 3)
            const bool two = h->opt.pipeline == 1 || h->opt.pipeline >= 4;
            PivotShape ps = choose_pipe_shape(h->prec, M, P, h->sms, h->opt.threads, h->opt.ctas,
                                              two ? 3 : 1);
            if (ps.pipe) {
                ps.pipe = two ? 3 : 2;
                if (two) ps.sel_warps = tbytes < kBlockBytes ? 8 : 4;
                return ps;
            }
        }
        return choose_shape(h->prec, rule, M, N, P, h->sms, h->opt.threads, h->opt.ctas);
    };
    const PivotShape sh = shape_for((int)sense);
    // the other rule (FP32 recovery, Phase 1 of Phase I)
    const PivotShape sh_alt = shape_for(1 - (int)sense);
    const bool two_rules = h->prec == PREC_FP32 || phase1;
    const int ctas_max = two_rules ? std::max(sh.ctas, sh_alt.ctas) : sh.ctas;

    CUDA_TRY(h, grow_bytes(h, &h->dT, &h->cap_T, (size_t)M * P * esz));
    CUDA_TRY(h, grow(h, &h->dbasis, &h->cap_basis, (size_t)m));
    {
        size_t need = sh.use_smem ? 0 : (size_t)sh.ctas * (size_t)sh.scratch_stride;
        if (two_rules && !sh_alt.use_smem)
            need = std::max(need, (size_t)sh_alt.ctas * (size_t)sh_alt.scratch_stride);
        if (need) CUDA_TRY(h, grow_bytes(h, &h->dscratch, &h->cap_scratch, need));
    }
    if (h->max_ctas < ctas_max) {
        dev_free(h, h->dpart);
        h->dpart = nullptr;
        h->max_ctas = 0;
        // records: 4 x G pricing candidates, then (in 8-byte words) 32 x G
        // record values, 16 x G ratio records, 4 x G exact candidates and
        // 16 x G exact values
        CUDA_TRY(h, dev_alloc(h, (void **)&h->dpart, 38 * (size_t)ctas_max * sizeof(Cand)));
        h->max_ctas = ctas_max;
    }
    if (h->opt.trace_cap > 0 && h->cap_trace < h->opt.trace_cap) {
        dev_free(h, h->dtrace);
        h->dtrace = nullptr;
        h->cap_trace = 0;
        CUDA_TRY(h, dev_alloc(h, (void **)&h->dtrace, 2 * (size_t)h->opt.trace_cap * sizeof(int)));
        h->cap_trace = h->opt.trace_cap;
    }
    CUDA_TRY(h, grow(h, &h->dx, &h->cap_x, (size_t)n));
    CUDA_TRY(h, grow(h, &h->dy, &h->cap_y, (size_t)m));

    cudaStream_t s = h->stream;
    const double amax = bits_to_double(st.amax_bits), bmax = bits_to_double(st.bmax_bits),
                 cmax = bits_to_double(st.cmax_bits);
    h->eps_d = h->opt.eps_d > 0 ? h->opt.eps_d : 1e-9 * std::max(1.0, cmax);
    h->eps_p = h->opt.eps_p > 0 ? h->opt.eps_p : 1e-9 * std::max(1.0, amax);
    h->eps_r = h->opt.eps_r > 0 ? h->opt.eps_r : 1e-9 * std::max(1.0, bmax);

    // FP32 tableau: the same tolerances as FP64.  A coarser pivot tolerance is
    // wrong here: entries of the basis-inverse (slack) columns scale like
    // 1/|A|, so a tolerance scaled by max|A| at FP32 resolution (1e-6) drops
    // legitimate pivot rows and leads the FP32 run to an infeasible basis.
    h->eps32_d = h->eps_d;
    h->eps32_p = h->eps_p;
    h->eps32_r = h->eps_r;
    if (h->prec == PREC_FP32 && h->cap_rb < (size_t)(m > n ? m : n) + m) {
        const size_t cap = (size_t)(m > n ? m : n) + m;
        void **ints[] = {(void **)&h->rb.Lflag, (void **)&h->rb.S, (void **)&h->rb.R,
                         (void **)&h->rb.posS, (void **)&h->rb.posR, (void **)&h->rb.pivrow};
        for (void **q : ints) {
            dev_free(h, *q);
            *q = nullptr;
            CUDA_TRY(h, dev_alloc(h, q, cap * sizeof(int)));
        }
        void **dbl[] = {(void **)&h->rb.xS, (void **)&h->rb.yR, (void **)&h->rb.zrow,
                        (void **)&h->rb.rhs};
        for (void **q : dbl) {
            dev_free(h, *q);
            *q = nullptr;
            CUDA_TRY(h, dev_alloc(h, q, cap * sizeof(double)));
        }
        if (!h->rb.counts) CUDA_TRY(h, dev_alloc(h, (void **)&h->rb.counts, 4 * sizeof(int)));
        if (!h->rb.chk) CUDA_TRY(h, dev_alloc(h, (void **)&h->rb.chk, sizeof(ReinvCheck)));
        if (!h->rb.bar) CUDA_TRY(h, dev_alloc(h, (void **)&h->rb.bar, 128 * sizeof(unsigned)));
        h->cap_rb = cap;
    }

    CUDA_TRY(h, launch_build(h->prec, h->dA, h->db, h->dc, m, n, phase1 ? 2 : (int)sense, h->dT, P,
                             h->dbasis, s));

    LpDesc d{};
    d.T = h->dT;
    d.basis = h->dbasis;
    d.scratch = h->dscratch;
    d.scratch_stride = sh.scratch_stride;
    d.part_sel = h->dpart;
    d.part_vals = reinterpret_cast<unsigned long long *>(h->dpart + 4 * (size_t)h->max_ctas);
    d.T2 = have_t2 ? h->dT2 : nullptr;
    d.colx = h->dcolx;
    d.abort = h->dabort;
    d.work = reinterpret_cast<unsigned long long *>(h->dbar + kBarWords);
    CUDA_TRY(h, cudaMemsetAsync(d.work, 0, 2 * sizeof(unsigned long long), s));
    // a constraint row may hold a -0: from the data, after Phase 1 (dual
    // pivots are negative), or in FP32 mode once a reinversion has rewritten
    // the rows (its refreshes and its dual-rule recovery; reinvert marks the
    // LP); the two-pivot primal kernel then starts each launch by finding the
    // vectors that do
    d.negz = (st.flags & 8) || phase1 ? 1 : 0;
    d.bar = h->dbar;
    d.err = (int *)(h->dbar + 96);
    d.trace = h->dtrace;
    d.trace_cap = h->opt.trace_cap > 0 ? h->opt.trace_cap : 0;
    d.P = P;
    d.m = m;
    d.n = n;
    d.M = M;
    d.N = N;
    d.sense = (int)sense;
    d.bland_after = h->opt.bland_after;
    d.eps_d = h->prec == PREC_FP64 ? h->eps_d : h->eps32_d;
    d.eps_p = h->prec == PREC_FP64 ? h->eps_p : h->eps32_p;
    d.eps_r = h->prec == PREC_FP64 ? h->eps_r : h->eps32_r;
    d.iters = 0;
    d.iter_limit = 0;
    d.deg = 0;
    d.status = -1;
    d.last_p = d.last_q = -1;
    CUDA_TRY(h, cudaMemcpyAsync(h->ddesc, &d, sizeof d, cudaMemcpyHostToDevice, s));
    *h->pdesc = d;
    h->desc = d;
    h->shape = sh;
    h->shape_alt = sh_alt;
    h->m = m;
    h->n = n;
    h->M = M;
    h->N = N;
    h->P = P;
    h->sense = (int)sense;
    h->phase = phase1 ? 1 : 0;
    h->loaded = true;
    return LP_OK;
}

}  // extern "C"

namespace {

// Start the wall-clock limit of a solve: lower the abort word (no kernel of
// this handle is running: the previous solve was waited for) and set the
// deadline.
void arm_deadline(lp_handle *h) {
    __atomic_store_n(h->habort, 0, __ATOMIC_SEQ_CST);
    if (h->opt.time_limit_s > 0.0)
        h->deadline = std::chrono::steady_clock::now() +
                      std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                          std::chrono::duration<double>(h->opt.time_limit_s));
}

bool past_deadline(const lp_handle *h) {
    return h->opt.time_limit_s > 0.0 && std::chrono::steady_clock::now() >= h->deadline;
}

// Wait for the handle's stream.  Under a wall-clock limit the host polls the
// stream and, once the deadline has passed, raises the abort word, which
// every pivot kernel reads once per pass: the kernel stops within a pass
// with status LP_TIMEOUT and the wait ends.
cudaError_t wait_stream(lp_handle *h) {
    if (h->opt.time_limit_s <= 0.0) return cudaStreamSynchronize(h->stream);
    bool raised = false;
    for (;;) {
        const cudaError_t e = cudaStreamQuery(h->stream);
        if (e != cudaErrorNotReady) return e;
        if (!raised && past_deadline(h)) {
            __atomic_store_n(h->habort, 1, __ATOMIC_SEQ_CST);
            raised = true;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// The double-buffered kernel leaves its last tableau in either buffer and
// names it in the descriptor; once the descriptor is read back, make it h->dT.
void adopt_tableau(lp_handle *h) {
    if (h->pdesc->T != h->dT && h->pdesc->T == h->dT2) {
        std::swap(h->dT, h->dT2);
        std::swap(h->cap_T, h->cap_T2);
    }
}

double okey_to_double(unsigned long long k) {
    const unsigned long long bits = (k & 0x8000000000000000ull) ? (k & ~0x8000000000000000ull) : ~k;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}

// FP64 reinversion of the current basis (gbs_reinv.cu); *zmin and *rmin
// receive the smallest FP64 objective-row entry and rhs.
lp_err reinvert(lp_handle *h, bool *singular, double *zmin, double *rmin) {
    cudaStream_t s = h->stream;
    const int m = h->m, n = h->n;
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    CUDA_TRY(h, cudaEventRecord(e0, s));
    CUDA_TRY(h, launch_reinv_lists(h->dbasis, m, n, h->rb, s));
    int counts[2] = {0, 0};
    CUDA_TRY(h, cudaMemcpyAsync(counts, h->rb.counts, sizeof counts, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    const int ns = counts[0];
    if (counts[1] != ns) {
        set_err(h, "reinversion: inconsistent basis (%d structural, %d free rows)", counts[0],
                counts[1]);
        return LP_ERR_STATE;
    }
    h->rb.Wp = ((long long)2 * ns + 1 + 31) / 32 * 32;
    const size_t need = (size_t)ns * (size_t)h->rb.Wp;
    if (need > h->cap_W) {
        dev_free(h, h->rb.W);
        h->rb.W = nullptr;
        h->cap_W = 0;
        // from a range (never freed), the largest this LP can need, at once
        const size_t nsx = (size_t)std::min(m, n);
        const size_t want = h->region ? std::max(need, nsx * ((2 * nsx + 1 + 31) / 32 * 32)) : need;
        CUDA_TRY(h, dev_alloc(h, (void **)&h->rb.W, std::max<size_t>(want, 1) * sizeof(double)));
        h->cap_W = want;
    }
    CUDA_TRY(h, launch_reinv_solve(h->prec, h->dA, h->db, h->dc, h->sense, m, n, h->dbasis, h->rb,
                                   ns, h->dT, h->P, h->dx, h->dy, h->dobj, h->sms,
                                   h->opt.spin_timeout_cycles, s));
    // the rows are rewritten from here on (rhs, objective row, the body's
    // refresh, the dual rule's recovery): a -0 may be present
    const int negz = 1;
    CUDA_TRY(h, cudaMemcpyAsync((char *)h->ddesc + offsetof(LpDesc, negz), &negz, sizeof negz,
                                cudaMemcpyHostToDevice, s));
    ReinvCheck chk;
    CUDA_TRY(h, cudaMemcpyAsync(&chk, h->rb.chk, sizeof chk, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaEventRecord(e1, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    float t = 0.0f;
    cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->reinv_ms += t;
    h->last_ns = ns;
    h->reinversions += 1;
    *singular = chk.singular != 0;
    *zmin = okey_to_double(chk.zmin_key);
    *rmin = okey_to_double(chk.rhsmin_key);
    return LP_OK;
}

// The FP32 tableau's constraint rows B^-1 [A I] recomputed from the FP64 data
// for the basis of the last reinversion (lp_options.reinv_body), before the
// tableau is pivoted again.
lp_err refresh_body(lp_handle *h) {
    if (h->prec != PREC_FP32 || !h->opt.reinv_body || h->region) return LP_OK;
    cudaStream_t s = h->stream;
    cudaEvent_t e0, e1;
    CUDA_TRY(h, cudaEventCreate(&e0));
    CUDA_TRY(h, cudaEventCreate(&e1));
    CUDA_TRY(h, cudaEventRecord(e0, s));
    CUDA_TRY(h, oz_refresh_body(h->dA, h->db, h->sense, h->m, h->n, h->dbasis, h->rb, h->last_ns,
                                static_cast<float *>(h->dT), h->P, h->oz, h->sms,
                                h->opt.spin_timeout_cycles, s));
    int oerr = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&oerr, h->oz.err, sizeof oerr, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaEventRecord(e1, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    float tb = 0.0f;
    cudaEventElapsedTime(&tb, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->reinv_ms += tb;
    h->body_ms += tb;
    if (oerr) {
        set_err(h, "reinversion: a wait of the body refresh ran out");
        return LP_ERR_CUDA;
    }
    return LP_OK;
}

// FP32 tableau with FP64 reinversion: pivot reinv_k pivots at a time in FP32,
// reinvert in FP64 after each batch and at termination; an FP32 optimum is
// accepted only when the FP64 values show it primal and dual feasible.
lp_err solve_fp32(lp_handle *h) {
    cudaStream_t s = h->stream;
    long long remaining = h->opt.max_iters;
    // Guard against FP32 runs that stop making progress: at most this many
    // pivots per solve call before LP_NUMERICAL.
    long long guard = 20ll * (h->m + h->n) + 1000;
    int failed_checks = 0;
    int rule = h->sense;  // 0: primal simplex, 1: dual simplex
    lp_status final = LP_NOT_SOLVED;
    h->fp32_kernel_ms = 0.0;
    h->fp32_launches = 0;
    h->reinv_ms = 0.0;
    h->body_ms = 0.0;
    h->reinversions = 0;
    for (;;) {
        const PivotShape &sh = rule == h->sense ? h->shape : h->shape_alt;
        const long long budget = std::min<long long>(remaining, (long long)h->opt.reinv_k);
        const long long before = h->pdesc->iters;
        const long long stride = sh.scratch_stride;
        CUDA_TRY(h, cudaMemcpyAsync((char *)h->ddesc + offsetof(LpDesc, scratch_stride), &stride,
                                    sizeof stride, cudaMemcpyHostToDevice, s));
        CUDA_TRY(h, cudaMemsetAsync(h->dbar, 0, kBarWords * sizeof(unsigned), s));
        CUDA_TRY(h, cudaEventRecord(h->ev0, s));
        CUDA_TRY(h, launch_pivot(h->prec, h->ddesc, sh, h->opt.spin_timeout_cycles, budget, s));
        CUDA_TRY(h, cudaEventRecord(h->ev1, s));
        CUDA_TRY(h, cudaMemcpyAsync(h->pdesc, h->ddesc, sizeof(LpDesc), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, wait_stream(h));
        adopt_tableau(h);
        float t = 0.0f;
        cudaEventElapsedTime(&t, h->ev0, h->ev1);
        h->fp32_kernel_ms += t;
        h->fp32_launches += 1;
        remaining -= h->pdesc->iters - before;
        guard -= h->pdesc->iters - before;
        const int st = h->pdesc->status;
        if (st == LP_TIMEOUT || past_deadline(h)) {
            final = LP_TIMEOUT;
            break;
        }
        bool singular = false;
        double zmin = 0.0, rmin = 0.0;
        lp_err e = reinvert(h, &singular, &zmin, &rmin);
        if (e != LP_OK) return e;
        if (singular) {
            final = LP_NUMERICAL;
            break;
        }
        const bool pfeas = rmin >= -h->eps_r, dfeas = zmin >= -h->eps_d;
        if (st == LP_OPTIMAL) {
            if (pfeas && dfeas) {
                final = LP_OPTIMAL;
                break;
            }
            if ((!pfeas && !dfeas) || ++failed_checks > 4) {
                final = LP_NUMERICAL;
                break;
            }
            // The FP32 run stopped at a basis the FP64 values reject.  From a
            // dual-feasible basis the dual simplex restores primal
            // feasibility, from a primal-feasible one the primal simplex
            // restores optimality; price with the FP64 tolerances on the
            // refreshed rhs and objective row.
            rule = pfeas ? 0 : 1;
            const double eps[3] = {h->eps_d, h->eps_p, h->eps_r};
            CUDA_TRY(h, cudaMemcpyAsync((char *)h->ddesc + offsetof(LpDesc, eps_d), eps,
                                        sizeof eps, cudaMemcpyHostToDevice, s));
            if ((e = refresh_body(h)) != LP_OK) return e;
            continue;
        }
        if (st == LP_UNBOUNDED || st == LP_INFEASIBLE) {
            final = (lp_status)st;
            break;
        }
        if (remaining <= 0) {  // ITER_LIMIT: a later lp_solve pivots on from here
            if ((e = refresh_body(h)) != LP_OK) return e;
            final = LP_ITER_LIMIT;
            break;
        }
        if (guard <= 0) {
            final = LP_NUMERICAL;
            break;
        }
        // periodic reinversion: when the FP64 values show the current rule's
        // invariant lost (primal simplex: feasible rhs; dual simplex:
        // nonnegative reduced costs) and the other rule's invariant holding,
        // continue with the other rule
        if (rule == 0 && !pfeas && dfeas) rule = 1;
        else if (rule == 1 && !dfeas && pfeas) rule = 0;
        if ((e = refresh_body(h)) != LP_OK) return e;
    }
    h->pdesc->status = final;
    if (final == LP_TIMEOUT) h->timed_out = true;
    CUDA_TRY(h, cudaMemcpyAsync(h->pobj, h->dobj, sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    h->solved = true;
    return LP_OK;
}

}  // namespace

extern "C" {

lp_err lp_solve_async(lp_handle *h) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->loaded) {
        set_err(h, "lp_solve: no LP loaded");
        return LP_ERR_STATE;
    }
    if (h->timed_out) {
        set_err(h, "lp_solve: the last solve ended in LP_TIMEOUT and left the tableau "
                   "undefined; load the LP again");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    arm_deadline(h);
    if (h->prec == PREC_FP32) return solve_fp32(h);
    cudaStream_t s = h->stream;
    // The pivot state (iterations, degeneracy counter) lives in the device
    // descriptor, so consecutive calls resume without a host round trip.
    long long budget = h->opt.max_iters;
    CUDA_TRY(h, cudaEventRecord(h->ev0, s));
    if (h->phase == 1) {
        // Phase I, Phase 1: the dual simplex rule on the tableau whose
        // objective row is max(-c, 0), until no rhs is below -eps_r.  The
        // host waits for its end to choose what follows.
        const long long before = h->pdesc->iters;
        CUDA_TRY(h, cudaMemsetAsync(h->dbar, 0, kBarWords * sizeof(unsigned), s));
        CUDA_TRY(h, launch_pivot(h->prec, h->ddesc, h->shape_alt, h->opt.spin_timeout_cycles,
                                 budget, s));
        CUDA_TRY(h, cudaMemcpyAsync(h->pdesc, h->ddesc, sizeof(LpDesc), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(h, wait_stream(h));
        adopt_tableau(h);
        if (h->pdesc->status == ST_OPTIMAL && !past_deadline(h)) {
            // Phase 2 from this basis: the objective row of c, the
            // degenerate-pivot count restarted
            CUDA_TRY(h, launch_phase2_objective(h->ddesc, h->dc, h->N, s));
            const int zero = 0;
            CUDA_TRY(h, cudaMemcpyAsync((char *)h->ddesc + offsetof(LpDesc, deg), &zero, sizeof zero,
                                        cudaMemcpyHostToDevice, s));
            h->phase = 2;
            budget -= h->pdesc->iters - before;
        } else {
            // infeasible (or stopped: iteration limit, timeout; resumable in
            // Phase 1 after the iteration limit)
            if (h->pdesc->status == ST_OPTIMAL) {  // Phase 1 done, but past the deadline
                h->pdesc->status = LP_TIMEOUT;
                const int st = LP_TIMEOUT;
                CUDA_TRY(h, cudaMemcpyAsync((char *)h->ddesc + offsetof(LpDesc, status), &st,
                                            sizeof st, cudaMemcpyHostToDevice, s));
            }
            CUDA_TRY(h, cudaEventRecord(h->ev1, s));
            CUDA_TRY(h, launch_extract(h->prec, h->ddesc, h->dT, h->dbasis, h->m, h->n, h->P,
                                       h->sense, h->dx, h->dy, h->dobj, s));
            CUDA_TRY(h, cudaMemcpyAsync(h->pobj, h->dobj, sizeof(double), cudaMemcpyDeviceToHost, s));
            h->solved = true;
            return LP_OK;
        }
    }
    CUDA_TRY(h, cudaMemsetAsync(h->dbar, 0, kBarWords * sizeof(unsigned), s));
    CUDA_TRY(h, launch_pivot(h->prec, h->ddesc, h->shape, h->opt.spin_timeout_cycles, budget, s));
    CUDA_TRY(h, cudaEventRecord(h->ev1, s));
    CUDA_TRY(h, launch_extract(h->prec, h->ddesc, h->dT, h->dbasis, h->m, h->n, h->P, h->sense,
                               h->dx, h->dy, h->dobj, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->pdesc, h->ddesc, sizeof(LpDesc), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaMemcpyAsync(h->pobj, h->dobj, sizeof(double), cudaMemcpyDeviceToHost, s));
    h->solved = true;
    return LP_OK;
}

lp_err lp_solve(lp_handle *h) {
    lp_err e = lp_solve_async(h);
    if (e != LP_OK) return e;
    CUDA_TRY(h, wait_stream(h));
    if (h->pdesc->status == LP_TIMEOUT) h->timed_out = true;
    return LP_OK;
}

lp_err lp_result(lp_handle *h, double *x, double *y, double *obj, lp_status *status,
                 long long *iters) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->solved) {
        set_err(h, "lp_result: nothing solved");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    CUDA_TRY(h, wait_stream(h));
    if (h->pdesc->status == LP_TIMEOUT) h->timed_out = true;
    if (x) CUDA_TRY(h, cudaMemcpyAsync(x, h->dx, sizeof(double) * h->n, cudaMemcpyDefault, s));
    if (y) CUDA_TRY(h, cudaMemcpyAsync(y, h->dy, sizeof(double) * h->m, cudaMemcpyDefault, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    if (obj) *obj = *h->pobj;
    if (status) *status = (lp_status)h->pdesc->status;
    if (iters) *iters = h->pdesc->iters;
    return LP_OK;
}

lp_err lp_update_counts(lp_handle *h, long long *updated, long long *in_place) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->loaded) {
        set_err(h, "lp_update_counts: no LP loaded");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, wait_stream(h));
    unsigned long long v[2] = {0ull, 0ull};
    CUDA_TRY(h, cudaMemcpy(v, h->dbar + kBarWords, sizeof v, cudaMemcpyDeviceToHost));
    // the kernels count vectors x pivots; a vector is 16 bytes of one row,
    // over the m constraint rows
    const long long per = (long long)(h->prec == PREC_FP64 ? 2 : 4) * h->m;
    if (updated) *updated = (long long)v[0] * per;
    if (in_place) *in_place = (long long)v[1] * per;
    return LP_OK;
}

lp_err lp_fp32_stats(lp_handle *h, int *reinversions, double *reinv_ms, double *body_ms) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (reinversions) *reinversions = h->reinversions;
    if (reinv_ms) *reinv_ms = h->reinv_ms;
    if (body_ms) *body_ms = h->body_ms;
    return LP_OK;
}

lp_err lp_kernel_time(lp_handle *h, double *ms, int *launches) {
    if (!h) return LP_ERR_INVALID_ARG;
    if (!h->solved) {
        set_err(h, "lp_kernel_time: nothing solved");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    if (h->prec == PREC_FP32) {
        if (ms) *ms = h->fp32_kernel_ms;
        if (launches) *launches = h->fp32_launches;
        return LP_OK;
    }
    CUDA_TRY(h, wait_stream(h));
    float t = 0.0f;
    CUDA_TRY(h, cudaEventElapsedTime(&t, h->ev0, h->ev1));
    if (ms) *ms = (double)t;
    if (launches) *launches = 1;
    return LP_OK;
}

lp_err lp_get_trace(lp_handle *h, int *rows, int *cols, long long cap, long long *count) {
    if (!h || cap < 0) return LP_ERR_INVALID_ARG;
    if (!h->loaded) {
        set_err(h, "lp_get_trace: no LP loaded");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    long long k = std::min(std::min(h->pdesc->iters, h->pdesc->trace_cap), cap);
    if (count) *count = k;
    if (k <= 0) return LP_OK;
    int *tmp = new (std::nothrow) int[2 * k];
    if (!tmp) return LP_ERR_OOM;
    cudaError_t e = cudaMemcpy(tmp, h->dtrace, sizeof(int) * 2 * k, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        delete[] tmp;
        set_err(h, "lp_get_trace: %s", cudaGetErrorString(e));
        return LP_ERR_CUDA;
    }
    for (long long i = 0; i < k; ++i) {
        if (rows) rows[i] = tmp[2 * i];
        if (cols) cols[i] = tmp[2 * i + 1];
    }
    delete[] tmp;
    return LP_OK;
}

lp_err lp_get_basis(lp_handle *h, int *basis) {
    if (!h || !basis) return LP_ERR_INVALID_ARG;
    if (!h->loaded) {
        set_err(h, "lp_get_basis: no LP loaded");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, cudaMemcpyAsync(basis, h->dbasis, sizeof(int) * h->m, cudaMemcpyDefault, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return LP_OK;
}

lp_err lp_get_tableau(lp_handle *h, double *T) {
    if (!h || !T) return LP_ERR_INVALID_ARG;
    if (!h->loaded) {
        set_err(h, "lp_get_tableau: no LP loaded");
        return LP_ERR_STATE;
    }
    DeviceRestore restore_;
    CUDA_TRY(h, cudaSetDevice(h->device));
    cudaStream_t s = h->stream;
    CUDA_TRY(h, cudaStreamSynchronize(s));
    adopt_tableau(h);
    if (h->prec == PREC_FP64) {
        CUDA_TRY(h, cudaMemcpy2DAsync(T, sizeof(double) * h->N, h->dT, sizeof(double) * h->P,
                                      sizeof(double) * h->N, h->M, cudaMemcpyDefault, s));
    } else {
        double *tmp = nullptr;
        CUDA_TRY(h, cudaMalloc(&tmp, sizeof(double) * (size_t)h->M * h->N));
        cudaError_t e = launch_to_fp64((const float *)h->dT, h->P, h->M, h->N, tmp, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(T, tmp, sizeof(double) * (size_t)h->M * h->N, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(tmp);
        if (e != cudaSuccess) {
            set_err(h, "lp_get_tableau: %s", cudaGetErrorString(e));
            return LP_ERR_CUDA;
        }
    }
    CUDA_TRY(h, cudaStreamSynchronize(s));
    return LP_OK;
}

}  // extern "C"

namespace gbs {

lp_err handle_bind_region(lp_handle *h, void *base, size_t bytes) {
    if (!h) {
        set_err(h, "handle_bind_region: NULL handle");
        return LP_ERR_INVALID_ARG;
    }
    DeviceRestore restore_;
    cudaSetDevice(h->device);
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    void **bufs[] = {(void **)&h->dA, (void **)&h->db, (void **)&h->dc, &h->dT, &h->dT2,
                     &h->dcolx, (void **)&h->dbasis, &h->dscratch, (void **)&h->dpart,
                     (void **)&h->dtrace, (void **)&h->dx, (void **)&h->dy,
                     (void **)&h->rb.Lflag, (void **)&h->rb.S, (void **)&h->rb.R,
                     (void **)&h->rb.posS, (void **)&h->rb.posR, (void **)&h->rb.counts,
                     (void **)&h->rb.pivrow, (void **)&h->rb.W, (void **)&h->rb.xS,
                     (void **)&h->rb.yR, (void **)&h->rb.zrow, (void **)&h->rb.rhs,
                     (void **)&h->rb.chk, (void **)&h->rb.bar};
    for (void **p : bufs) {
        dev_free(h, *p);
        *p = nullptr;
    }
    h->cap_A = h->cap_b = h->cap_c = h->cap_T = h->cap_T2 = h->cap_colx = 0;
    h->cap_basis = h->cap_scratch = h->cap_x = h->cap_y = 0;
    h->max_ctas = 0;
    h->cap_trace = 0;
    h->cap_W = h->cap_rb = 0;
    h->loaded = h->solved = false;
    h->region = static_cast<unsigned char *>(base);
    h->region_size = base ? bytes : 0;
    h->region_used = 0;
    return LP_OK;
}

size_t handle_region_used(const lp_handle *h) { return h ? h->region_used : 0; }

void handle_set_max_iters(lp_handle *h, long long n) {
    if (h) h->opt.max_iters = n;
}

}  // namespace gbs
