// Allocation-free solve: lp_solve_noalloc (declared in include/gbsimplex.h).
//
// Some callers cannot allocate device memory at the point where they want to
// solve an LP: code that runs with a fixed device-memory budget handed out up
// front, plug-ins hosted by a process that owns the allocator, or real-time
// loops that must not hit cudaMalloc's latency.  For them this file keeps all
// working memory of one FP64 solve -- the tableau, the input copies, the basis,
// the per-CTA partials, the barrier words and the results -- in one
// file-scope device array of fixed size.  Every GPU that loads the library
// holds that array until the process exits.
//
// The array is shared by every call in the process: each call rebuilds what it
// reads (tableau, basis, partials) and clears the barrier words, so stale
// contents of an earlier call never leak into a result.  Calls are serialised
// by a host mutex and each call waits for its own work before returning; work
// from this entry point that overlapped on the GPU (for example from two
// processes sharing one context) would race on the array.
//
// Set-up: the first call on a device, with that device current, looks up the
// array's device address with cudaGetSymbolAddress (in host code the array's
// name is only a host-side stand-in) and caches it per device.  Make that first
// call before any stream capture.
//
// The solve runs the one-pivot in-place kernel (pivot_kernel: selection, then
// the update, one grid barrier per pivot), whose per-launch state is the
// 2 x CTAs pricing partials and the barrier block; the pipelined kernels need
// more record space and a second tableau, which this array does not hold.

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "gbs_internal.h"
#include "gbsimplex.h"

using namespace gbs;

namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[kMaxDevices] = {nullptr};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Errors are reported like lp_create's: the message is lp_last_error(NULL).
lp_err fail(lp_err code, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error_global(msg);
    return code;
}

struct Layout {
    size_t desc, stats, bar, part, basis, A, b, c, x, y, obj, T, scratch, total;
};

Layout layout_for(int m, int n, long long P, const PivotShape &sh) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off += up256(bytes);
        return at;
    };
    const int M = m + 1;
    L.desc = take(sizeof(LpDesc));
    L.stats = take(sizeof(InputStats));
    L.bar = take(kBarWords * sizeof(unsigned));
    L.part = take(2 * (size_t)sh.ctas * sizeof(Cand));  // pivot_kernel's partials (sh.pipe == 0)
    L.basis = take((size_t)m * sizeof(int));
    L.A = take((size_t)m * n * sizeof(double));
    L.b = take((size_t)m * sizeof(double));
    L.c = take((size_t)n * sizeof(double));
    L.x = take((size_t)n * sizeof(double));
    L.y = take((size_t)m * sizeof(double));
    L.obj = take(sizeof(double));
    L.T = take((size_t)M * (size_t)P * sizeof(double));
    L.scratch = take(sh.use_smem ? 0 : (size_t)sh.ctas * (size_t)sh.scratch_stride);
    L.total = off;
    return L;
}

// Waits for the caller's stream on every return once this call has queued
// work there, so that the lock on the shared array is released only when no
// copy or kernel of this call can still touch it (declared after the lock,
// so it runs first).
struct DrainStream {
    cudaStream_t s;
    bool armed = false;
    explicit DrainStream(cudaStream_t st) : s(st) {}
    ~DrainStream() {
        if (armed) cudaStreamSynchronize(s);
    }
};

}  // namespace

#define NA_TRY(call)                                                                  \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(LP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

extern "C" lp_err lp_solve_noalloc(int m, int n, const double *A, const double *b,
                                   const double *c, lp_sense sense, const lp_options *opt,
                                   double *x, double *y, double *obj, lp_status *status,
                                   long long *iters) {
    if (m < 1 || n < 1 || !A || !b || !c)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: need m, n >= 1 and non-NULL A, b, c");
    if (sense != LP_MAX_LE && sense != LP_MIN_GE)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: unknown sense %d", (int)sense);
    lp_options o;
    if (opt) o = *opt; else lp_options_default(&o);
    if (o.precision != LP_FP64)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: FP64 only");
    if (o.max_iters < 0 || o.bland_after < 0 || o.spin_timeout_cycles <= 0 || o.threads < 0 ||
        o.threads > 1024 || o.ctas < 0)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: option out of range");
    if ((long long)n + m + 1 > 0x7fffffffll - 64)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: n + m too large");
    if (o.device < 0 || o.device >= kMaxDevices)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: device %d out of range", o.device);

    DeviceRestore restore;
    NA_TRY(cudaSetDevice(o.device));
    int sms = 0;
    NA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device));
    const int M = m + 1, N = n + m + 1;
    const long long P = pitch_for(N);
    const PivotShape sh = choose_shape(PREC_FP64, (int)sense, M, N, P, sms, o.threads, o.ctas);
    if (sh.pipe != 0)  // the layout holds pivot_kernel's state only
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: internal: pipelined shape");
    const Layout L = layout_for(m, n, P, sh);
    if (L.total > kNoAllocBytes)
        return fail(LP_ERR_INVALID_ARG,
                    "lp_solve_noalloc: a %d x %d LP needs %zu bytes of working memory; this entry "
                    "point holds %zu (64 MiB)", m, n, L.total, kNoAllocBytes);

    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[o.device]) {
        void *ptr = nullptr;
        NA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_ptr[o.device] = ptr;
    }
    unsigned char *base = static_cast<unsigned char *>(g_noalloc_ptr[o.device]);
    LpDesc *d_desc = reinterpret_cast<LpDesc *>(base + L.desc);
    InputStats *d_stats = reinterpret_cast<InputStats *>(base + L.stats);
    unsigned *d_bar = reinterpret_cast<unsigned *>(base + L.bar);
    double *dA = reinterpret_cast<double *>(base + L.A);
    double *db = reinterpret_cast<double *>(base + L.b);
    double *dc = reinterpret_cast<double *>(base + L.c);
    double *dx = reinterpret_cast<double *>(base + L.x);
    double *dy = reinterpret_cast<double *>(base + L.y);
    double *dobj = reinterpret_cast<double *>(base + L.obj);
    int *dbasis = reinterpret_cast<int *>(base + L.basis);
    void *dT = base + L.T;
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    DrainStream drain(s);
    drain.armed = true;

    NA_TRY(cudaMemcpyAsync(dA, A, sizeof(double) * (size_t)m * n, cudaMemcpyDefault, s));
    NA_TRY(cudaMemcpyAsync(db, b, sizeof(double) * (size_t)m, cudaMemcpyDefault, s));
    NA_TRY(cudaMemcpyAsync(dc, c, sizeof(double) * (size_t)n, cudaMemcpyDefault, s));
    NA_TRY(launch_inspect(dA, db, dc, m, n, d_stats, s));
    InputStats st;
    NA_TRY(cudaMemcpyAsync(&st, d_stats, sizeof st, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (st.flags & 4)
        return fail(LP_ERR_INVALID_ARG, "lp_solve_noalloc: A, b or c holds a NaN or infinity");
    if (sense == LP_MAX_LE && (st.flags & 1))
        return fail(LP_ERR_INFEASIBLE_START, "lp_solve_noalloc: max form needs b >= 0");
    if (sense == LP_MIN_GE && (st.flags & 2))
        return fail(LP_ERR_INFEASIBLE_START, "lp_solve_noalloc: min form needs c >= 0");
    double amax, bmax, cmax;
    memcpy(&amax, &st.amax_bits, sizeof amax);
    memcpy(&bmax, &st.bmax_bits, sizeof bmax);
    memcpy(&cmax, &st.cmax_bits, sizeof cmax);

    NA_TRY(launch_build(PREC_FP64, dA, db, dc, m, n, (int)sense, dT, P, dbasis, s));
    LpDesc d{};
    d.T = dT;
    d.basis = dbasis;
    d.scratch = sh.use_smem ? nullptr : base + L.scratch;
    d.scratch_stride = sh.scratch_stride;
    d.part_sel = reinterpret_cast<Cand *>(base + L.part);
    d.bar = d_bar;
    d.err = reinterpret_cast<int *>(d_bar + 96);
    d.trace = nullptr;
    d.trace_cap = 0;
    d.P = P;
    d.m = m;
    d.n = n;
    d.M = M;
    d.N = N;
    d.sense = (int)sense;
    d.bland_after = o.bland_after;
    d.eps_d = o.eps_d > 0 ? o.eps_d : 1e-9 * std::max(1.0, cmax);
    d.eps_p = o.eps_p > 0 ? o.eps_p : 1e-9 * std::max(1.0, amax);
    d.eps_r = o.eps_r > 0 ? o.eps_r : 1e-9 * std::max(1.0, bmax);
    d.iters = 0;
    d.deg = 0;
    d.status = -1;
    d.last_p = d.last_q = -1;
    NA_TRY(cudaMemcpyAsync(d_desc, &d, sizeof d, cudaMemcpyHostToDevice, s));
    // The barrier words and the timeout flag must start at zero.
    NA_TRY(cudaMemsetAsync(d_bar, 0, kBarWords * sizeof(unsigned), s));
    NA_TRY(launch_pivot(PREC_FP64, d_desc, sh, o.spin_timeout_cycles, o.max_iters, s));
    NA_TRY(launch_extract(PREC_FP64, d_desc, dT, dbasis, m, n, P, (int)sense, dx, dy, dobj, s));
    LpDesc out;
    double o_obj = 0.0;
    NA_TRY(cudaMemcpyAsync(&out, d_desc, sizeof out, cudaMemcpyDeviceToHost, s));
    NA_TRY(cudaMemcpyAsync(&o_obj, dobj, sizeof o_obj, cudaMemcpyDeviceToHost, s));
    if (x) NA_TRY(cudaMemcpyAsync(x, dx, sizeof(double) * (size_t)n, cudaMemcpyDefault, s));
    if (y) NA_TRY(cudaMemcpyAsync(y, dy, sizeof(double) * (size_t)m, cudaMemcpyDefault, s));
    NA_TRY(cudaStreamSynchronize(s));
    if (obj) *obj = o_obj;
    if (status) *status = (lp_status)out.status;
    if (iters) *iters = out.iters;
    return LP_OK;
}
