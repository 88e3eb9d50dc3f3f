// Internal interface between the C ABI (gbs_capi.cu) and the kernels
// (gbs_pivot.cu).  Not part of the public header.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "gbsimplex.h"

namespace gbs {

enum : int {
    ST_RUNNING = -1,
    ST_OPTIMAL = 0,
    ST_UNBOUNDED = 1,
    ST_ITER_LIMIT = 2,
    ST_INFEASIBLE = 3,
    ST_NUMERICAL = 4,
    ST_TIMEOUT = 5,
};

// A selection candidate: lexicographic minimum on (vk, key), where vk is an
// order-preserving integer image of the value compared; idx is the row or
// column it names, -1 for "no candidate".  Keys are unique within one
// selection, so the minimum is unique and independent of reduction order.
struct Cand {
    unsigned long long vk;
    int key;
    int idx;
};

// Device-resident description and state of one LP tableau.  Written by the
// host before a launch, updated by the pivot kernel, read back after it.
struct LpDesc {
    void *T;                   // M x P tableau (double or float), row-major, pitch P
    int *basis;                // basic variable of each constraint row (m)
    void *scratch;             // per-CTA selection scratch when shared memory is too small
    long long scratch_stride;  // bytes of scratch per CTA
    Cand *part_sel;            // 2 x G selection partials (pricing / leaving row), by parity
    unsigned *bar;             // [0] arrivals, [32] generation, [64] readers counter
    int *err;                  // set to 1 by a wait that timed out
    int *trace;                // 2 * trace_cap ints: (row, column) per pivot
    long long trace_cap;
    long long P;               // row pitch in elements (multiple of 32)
    int m, n, M, N;            // M = m + 1 rows, N = n + m + 1 columns
    int sense;                 // 0: primal simplex (max, <=); 1: dual simplex (min, >=)
    int bland_after;
    double eps_d, eps_p, eps_r;
    // state carried across launches
    long long iters;
    long long iter_limit;  // last launch stopped (ITER_LIMIT) once iters reached this
    int deg;               // consecutive zero-ratio pivots
    int status;
    int last_p, last_q;
    // batched launches: CTAs per LP and their column strip width
    int group, strip;
    // pipelined kernels: the second tableau buffer (double-buffered mode;
    // nullptr in place) and the values that come with the records (by
    // parity: the new pivot-row entries at the record's column and at the
    // rhs; 2 x G pairs, or 4 x G x 8 values for two pivots per pass)
    void *T2;
    unsigned long long *part_vals;
    // two-pivot primal kernel: the global slots of its four pivot columns
    // (4 x the column bytes rounded up to 16; the distributed ratio test
    // assembles each new column there)
    void *colx;
    // single-LP solves: the host's abort word (mapped host memory), nonzero
    // once the solve is past its wall-clock limit; nullptr elsewhere.  Each
    // pivot kernel reads it once per pass and ends in ST_TIMEOUT.
    const int *abort;
    // two-pivot primal kernel: vectors x pivots updated ([0]) and left in
    // place because both pivot rows are zero on them ([1]), added up over the
    // passes; nullptr: not counted
    unsigned long long *work;
    // nonzero when a constraint row may hold a -0 (from the data, Phase I,
    // FP32 mode, or a -0 an update produced): no vector is left in place
    int negz;
};

// Launch shape of the persistent pivot kernel for one LP.
struct PivotShape {
    int ctas = 0;                  // grid size (= number of column strips)
    int threads = 0;               // CTA size
    int strip = 0;                 // columns per strip (multiple of 32 bytes of elements)
    int use_smem = 0;              // selection scratch in shared memory (else global)
    int dual = 0;                  // dual simplex kernel (else primal)
    int pipe = 0;                  // pipelined kernel: 1 in place, 2 double-buffered, 3 two pivots per pass
    int sel_warps = 4;             // two pivots per pass: selection warps per CTA (4 or 8)
    int dist = 0;                  // two pivots per pass, primal: ratio test distributed over the CTAs
    int split = 0;                 // two pivots per pass, primal: first column of every CTA's second
                                   // run (0: one contiguous strip, every vector updated)
    size_t smem_bytes = 0;         // dynamic shared memory per CTA
    long long scratch_stride = 0;  // global scratch bytes per CTA when !use_smem
};

// Words of a pivot launch's synchronisation block (zeroed before each launch):
// [0] grid-barrier count, [32] its generation, [64] readers counter (in-place
// kernel) or pricing-records counter (pipelined kernel), [96] error flag,
// [128] selections-done counter (one-pivot pipelined kernels) or records
// counter (two-pivot dual kernel), [160] selections-done counter (two-pivot
// kernels), [192] ratio-records counter and [224] exact-rounds counter
// (two-pivot primal kernel); 128-byte apart.
constexpr int kBarWords = 256;

struct InputStats {
    unsigned long long amax_bits, bmax_bits, cmax_bits;  // bit patterns of max |.|
    int flags;  // 1: some b < 0, 2: some c < 0, 4: a non-finite value, 8: a -0 in A or b
    int pad_;
};

enum : int { PREC_FP64 = 0, PREC_FP32 = 1 };

// Launch limits of the persistent pivot kernels.
constexpr int kMaxThreads = 1024;
constexpr size_t kMaxDynSmem = 200 * 1024;  // below the 227 KB opt-in limit, leaving room for statics

inline long long pitch_for(int N) { return ((long long)N + 31) / 32 * 32; }

// Kernel launchers (gbs_pivot.cu).  All enqueue on `s` and return the launch
// status.
cudaError_t launch_inspect(const double *A, const double *b, const double *c, int m, int n,
                           InputStats *out, cudaStream_t s);
// sense 0 primal form, 1 dual form, 2 Phase 1 of Phase I (primal rows,
// objective row max(-c, 0))
cudaError_t launch_build(int prec, const double *A, const double *b, const double *c, int m,
                         int n, int sense, void *T, long long P, int *basis, cudaStream_t s);
// Phase I, the start of Phase 2 (FP64): the objective row of max c'x in the
// current basis, over the N columns of the tableau the descriptor names.
cudaError_t launch_phase2_objective(const LpDesc *d_desc, const double *c, int N, cudaStream_t s);
PivotShape choose_shape(int prec, int sense, int M, int N, long long P, int sms, int threads,
                        int ctas);
cudaError_t launch_pivot(int prec, LpDesc *d_desc, const PivotShape &sh, long long spin_limit,
                         long long budget, cudaStream_t s);
// Batched persistent launch over nitems (lp, rank) work items (gbs_pivot.cu).
cudaError_t launch_batch(int prec, LpDesc *descs, const int2 *items, int nitems, unsigned *queue,
                         int ctas, int threads, size_t smem, int use_smem, long long spin_limit,
                         long long budget, cudaStream_t s);
int max_coresident_batch_ctas(int prec, int threads, size_t smem, int use_smem, int sms);
// Pipelined primal kernel (selection of pivot k+1 overlapped with pivot k's update).
// The returned shape has pipe == 0 when the kernel cannot take the LP (a grid
// larger than one CTA per SM); its scratch is in shared memory when it fits,
// else a global slice of scratch_stride bytes per CTA.
// dual: 1 the dual simplex kernel, 2 the two-pivot primal kernel (both
// double-buffered only), 0 the primal kernel.
// split (two-pivot kernels, dual >= 2): the column where each CTA's second
// segment of columns starts, or 0; the shape keeps it only when every CTA's
// two segments fit its update threads.
PivotShape choose_pipe_shape(int prec, int M, long long P, int sms, int threads, int ctas,
                             int dual, int split = 0);
cudaError_t launch_pivot_pipe(int prec, LpDesc *d_desc, const PivotShape &sh,
                              long long spin_limit, long long budget, cudaStream_t s);
cudaError_t launch_extract(int prec, const LpDesc *d_desc, const void *T, const int *basis,
                           int m, int n, long long P, int sense, double *x, double *y,
                           double *obj, cudaStream_t s);
// Buffers of the FP64 reinversion (gbs_reinv.cu), owned by the handle.
struct ReinvCheck {
    unsigned long long zmin_key;    // okey of the smallest objective-row entry
    unsigned long long rhsmin_key;  // okey of the smallest rhs
    int singular;                   // the basis matrix had no pivot in some column
    int pad_;
};
struct ReinvBufs {
    int *Lflag, *S, *R, *posS, *posR, *counts, *pivrow;
    double *W;          // s x Wp Gauss-Jordan system [A_RS | b_R | I]
    long long Wp;
    double *xS, *yR, *zrow, *rhs;
    ReinvCheck *chk;
    unsigned *bar;      // barrier words for the Gauss-Jordan grid
};

cudaError_t launch_reinv_lists(const int *basis, int m, int n, const ReinvBufs &rb,
                               cudaStream_t s);

// One LP of a batched FP64 reinversion (gbs_reinv.cu): its data, tableau,
// outputs and slices of workspace.  The batched solve takes LPs with at most
// kReinvCtaMax structural basic variables, one CTA (1024 threads) each, with
// the arithmetic of the multi-CTA kernels, so the results are the same bits.
constexpr int kReinvCtaMax = 128;
struct ReinvItem {
    const double *A, *b, *c;
    int m, n, sense, ns;  // ns: structural basic variables (the lists pass's counts[0])
    const int *basis;
    void *T;
    long long P;
    double *x, *y, *obj;
    int *Lflag, *S, *R, *posS, *posR, *counts;
    double *W;
    long long Wp;
    double *xS, *yR, *zrow, *rhs;
    ReinvCheck *chk;
};
cudaError_t launch_reinv_lists_batch(const ReinvItem *d_items, int count, cudaStream_t s);
cudaError_t launch_reinv_solve_batch(int prec, const ReinvItem *d_items, int count, cudaStream_t s);

// One LP to reinvert: original FP64 data, its sense, basis, tableau and outputs.
struct ReinvJob {
    const double *A, *b, *c;
    int m, n, sense;
    const int *basis;
    void *T;
    long long P;
    double *x, *y, *obj;
};
struct ReinvPool;
// Grow-only workspace of reinvert_many (device slices per LP, pinned mirrors).
struct BatchReinv {
    int *d_int = nullptr, *d_counts = nullptr, *h_counts = nullptr;
    double *d_dbl = nullptr, *d_W = nullptr;
    ReinvItem *d_items = nullptr, *h_items = nullptr;
    ReinvCheck *d_chk = nullptr, *h_chk = nullptr;
    size_t cap_int = 0, cap_dbl = 0, cap_W = 0, cap_n = 0;
    ~BatchReinv();
};
// The FP64 reinversion of many LPs (gbs_reinv.cu): the lists of all in one
// launch, then every LP with at most kReinvCtaMax structural basics in one
// launch of a CTA each, the others one by one with the multi-CTA kernels
// (rp), the same bits either way.  On return ws.h_chk[k] is job k's check;
// *bad is the first job with an inconsistent basis, or -1.
cudaError_t reinvert_many(int prec, const ReinvJob *jobs, int count, BatchReinv &ws,
                          ReinvPool &rp, int sms, long long spin_limit, cudaStream_t s, int *bad);

// The double whose order-preserving key is k (the reinversion's check minima).
inline double key_to_double(unsigned long long k) {
    const unsigned long long bits = (k & 0x8000000000000000ull) ? (k & ~0x8000000000000000ull) : ~k;
    double d;
    memcpy(&d, &bits, sizeof d);
    return d;
}

// Device buffers of one FP64 reinversion, sized for the largest LP and reused
// LP by LP.
struct ReinvPool {
    ReinvBufs rb{};
    size_t cap_W = 0;
    int *h_counts = nullptr;
    ReinvCheck *h_chk = nullptr;
    ~ReinvPool() {
        void *bufs[] = {rb.Lflag, rb.S, rb.R, rb.posS, rb.posR, rb.counts, rb.pivrow, rb.W,
                        rb.xS, rb.yR, rb.zrow, rb.rhs, rb.chk, rb.bar};
        for (void *p : bufs)
            if (p) cudaFree(p);
        if (h_counts) cudaFreeHost(h_counts);
        if (h_chk) cudaFreeHost(h_chk);
    }
    cudaError_t init(size_t cap) {
        void **ints[] = {(void **)&rb.Lflag, (void **)&rb.S, (void **)&rb.R, (void **)&rb.posS,
                         (void **)&rb.posR, (void **)&rb.pivrow};
        for (void **q : ints) {
            cudaError_t e = cudaMalloc(q, cap * sizeof(int));
            if (e != cudaSuccess) return e;
        }
        void **dbl[] = {(void **)&rb.xS, (void **)&rb.yR, (void **)&rb.zrow, (void **)&rb.rhs};
        for (void **q : dbl) {
            cudaError_t e = cudaMalloc(q, cap * sizeof(double));
            if (e != cudaSuccess) return e;
        }
        cudaError_t e = cudaMalloc(&rb.counts, 4 * sizeof(int));
        if (e == cudaSuccess) e = cudaMalloc(&rb.chk, sizeof(ReinvCheck));
        if (e == cudaSuccess) e = cudaMalloc(&rb.bar, 128 * sizeof(unsigned));
        if (e == cudaSuccess) e = cudaMallocHost(&h_counts, 4 * sizeof(int));
        if (e == cudaSuccess) e = cudaMallocHost(&h_chk, sizeof(ReinvCheck));
        return e;
    }
};

// Everything after the lists, for ns structural basics (W sized for ns).
// Writes the FP64 solution (x, y, obj), the refreshed rhs column and
// objective row of T and the check minima.
cudaError_t launch_reinv_solve(int prec, const double *A, const double *b, const double *c,
                               int sense, int m, int n, const int *basis, const ReinvBufs &rb,
                               int ns, void *T, long long P, double *x, double *y, double *obj,
                               int sms, long long spin_limit, cudaStream_t s);

// ------------------------------------------------------------- serving --
// One admitted LP of the server (device memory, written by the host before
// the slot is marked ready).
struct ServeSlot {
    LpDesc d;                    // T, basis, partials, barrier words, sizes, group, strip
    const double *A, *b, *c;     // inputs copied to the device
    double *x, *y, *obj;         // outputs (device)
    InputStats *stats;           // zeroed by the host
    double opt_eps_d, opt_eps_p, opt_eps_r;  // > 0: caller's tolerances
    long long budget;            // pivot limit
};
constexpr int kServeQueue = 1 << 16;  // work-item ring
// Device-side control block of the server kernel.
struct ServeCtl {
    unsigned head;       // worker tickets taken
    unsigned tail;       // items published by the dispatcher
    int in_flight;       // slots dispatched and not yet completed
    int err;             // a bounded wait ran out
    int2 items[kServeQueue];
    unsigned seq[kServeQueue];  // item t is published when seq[t % Q] == t + 1
};
// Host-device ring in mapped pinned host memory.
constexpr int kServeMaxSlots = 4096;
struct ServeRing {
    int rq[kServeMaxSlots];    // slots made ready by the host, in order
    int rq_tail;               // host: entries of rq written
    int rq_head;               // dispatcher: entries of rq consumed
    int done[kServeMaxSlots];  // device: 1 = slot finished; host: back to 0
    int shutdown;              // host: exit as soon as idle
};
cudaError_t launch_server(ServeSlot *slots, int nslots, ServeCtl *ctl, ServeRing *ring_dev,
                          int ctas, int threads, size_t smem, long long spin_limit,
                          long long idle_limit, cudaStream_t s);
int max_coresident_server_ctas(int threads, size_t smem, int sms);

// Record the message returned by lp_last_error(NULL) (gbs_capi.cu).
void set_last_error_global(const char *msg);

// Make a handle take the device buffers that lp_load and the FP32 mode's
// reinversions size (inputs, tableaus, pivot-column slots, basis, scratch,
// records, trace, results, reinversion lists and matrix) from
// [base, base + bytes) instead of cudaMalloc: the server's solves of large
// LPs run on a handle bound to its HBM arena.  Waits for the
// handle's stream, drops its buffers (a cudaFree unless they came from a
// range) and marks it unloaded; base NULL unbinds.  The next lp_load carves
// from the start of the range and fails with LP_ERR_OOM when it is too
// small; handle_region_used reports the bytes taken so far.
lp_err handle_bind_region(lp_handle *h, void *base, size_t bytes);
size_t handle_region_used(const lp_handle *h);
// Pivots per lp_solve call of a handle (its lp_options.max_iters): the
// servers cut the solve of an LP that runs alone into slices with it.
void handle_set_max_iters(lp_handle *h, long long n);

cudaError_t launch_to_fp64(const float *T, long long P, int M, int N, double *out,
                           cudaStream_t s);

// Emulated-FP64 products on the tensor cores (gbs_ozaki.cu): device
// workspace, grown on demand and kept between calls.
struct OzWork {
    void *asl = nullptr, *bsl = nullptr;       // bf16 digit planes of A and B
    int *rowexp = nullptr, *colexp = nullptr;  // row / column exponents
    int *kx = nullptr;                         // inner exponents and balancing shifts
    int *pmask = nullptr;                      // nonzero digit planes per block
    size_t cap_asl = 0, cap_bsl = 0, cap_rowexp = 0, cap_colexp = 0, cap_kx = 0, cap_pmask = 0;
    // body refresh
    double *X = nullptr, *Ainv = nullptr, *Z = nullptr;
    int *basic_row = nullptr, *L = nullptr, *Lrow = nullptr;
    size_t cap_X = 0, cap_Ainv = 0, cap_Z = 0, cap_basic = 0, cap_L = 0, cap_Lrow = 0;
    int *err = nullptr;  // the product kernel's error flag (one int)
    unsigned long long *mmas = nullptr;  // tensor-core MMAs the last product issued
};
void oz_work_free(OzWork &w);

// C (M x N, ldc) = A (M x K, lda) B (K x N, ldb), FP64 in and out, all device
// memory, through bf16 digit products on the tensor cores.  *d_err (device)
// is set when a wait of the kernel ran out.
cudaError_t oz_dgemm(const double *A, long long lda, const double *B, long long ldb, double *C,
                     long long ldc, int M, int N, int K, OzWork &w, int *d_err, int sms,
                     long long spin_limit, cudaStream_t s);

// The FP32 tableau's constraint rows B^-1 [A I] (every column but the rhs),
// recomputed from the original data for the current basis, after the
// reinversion's lists and Gauss-Jordan step (rb, ns structural basics).
cudaError_t oz_refresh_body(const double *A, const double *b, int sense, int m, int n,
                            const int *basis, const ReinvBufs &rb, int ns, float *T32,
                            long long P, OzWork &w, int sms, long long spin_limit,
                            cudaStream_t s);

// Raise a kernel's dynamic shared memory limit (cudaFuncAttributeMax-
// DynamicSharedMemorySize, a per-function setting shared by every host
// thread) to the most the current device allows beside the kernel's static
// shared memory.  Every launch site sets this same value, so host threads
// that launch one kernel at once with different sizes (handles on different
// threads) never lower the limit under one another's launch.  The value per
// kernel and device is looked up once.
cudaError_t allow_dyn_smem(const void *fn);

// Host side: restores the caller's current device when an entry point that
// switched to its own device returns.
struct DeviceRestore {
    int dev = -1;
    DeviceRestore() {
        if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
    }
    ~DeviceRestore() {
        if (dev >= 0) cudaSetDevice(dev);
    }
    DeviceRestore(const DeviceRestore &) = delete;
    DeviceRestore &operator=(const DeviceRestore &) = delete;
};

}  // namespace gbs
