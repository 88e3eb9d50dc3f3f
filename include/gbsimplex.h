/*
 * gbsimplex -- dense tableau simplex on one GB300 (sm_103a), C ABI.
 *
 * The method is the standard tableau simplex of Coutinho et al., "A Scalable
 * Shared-Memory Parallel Simplex for Large-Scale Linear Programming"
 * (arXiv:1804.04737), Sec. 2 (Steps 1-5) and its parallel scheme of Sec. 3
 * (Steps I-VI), re-laid for a GPU: one persistent grid runs whole pivot
 * sequences; each pivot is Dantzig pricing (Sec. 2 Step 2), the ratio test
 * (Step 3) and the rank-1 tableau update (Steps 4-5).
 *
 * Problem forms (Sec. 2, Eq. 1 with m <= constraints and slack variables):
 *   LP_MAX_LE  max c'x  s.t. Ax <= b, x >= 0   (solved by the primal simplex
 *              from the slack basis, which b >= 0 makes feasible; with some
 *              b_i < 0, single FP64 solves go through Phase I, below)
 *   LP_MIN_GE  min c'x  s.t. Ax >= b, x >= 0   (needs c >= 0: the slack basis
 *              is dual feasible; solved by the dual simplex).  Loading
 *              (A', c, b) of a LP_MAX_LE problem in this form solves its LP
 *              dual, the "dual formulation" runs of Sec. 4.
 *
 * Arithmetic contract (FP64 mode), identical in the library and its test
 * oracle, so that pivot sequences agree bit for bit:
 *   pricing   candidate j < n+m with z_j < -eps_d; most negative wins, ties
 *             smallest j (Bland mode: smallest candidate j);
 *   ratio     rows with a_iq > eps_p; (rhs > 0 ? rhs : 0) / a_iq by one IEEE
 *             division; smallest wins, ties smallest row (Bland mode:
 *             smallest basic-variable index); none => LP_UNBOUNDED;
 *   pivot     prow_j = T[p][j] / T[p][q] (IEEE division), other rows
 *             T[i][j] = fma(-T[i][q], prow_j, T[i][j]), objective row too;
 *   Bland     after `bland_after` consecutive pivots whose chosen ratio is
 *             exactly 0, Bland's rule until the next nonzero ratio;
 *   dual      leaving row: most negative rhs below -eps_r (ties smallest
 *             row; Bland mode: smallest basic index); entering column: the
 *             smallest (z_j > 0 ? z_j : 0) / (-T[r][j]) over T[r][j] < -eps_p,
 *             ties smallest j; none => LP_INFEASIBLE;
 *   Phase I   (not in the paper; LP_MAX_LE with some b_i < 0, lp_load and
 *             lp_solve in FP64) Phase 1 builds the objective row
 *             [max(-c, 0) | 0 | 0], dual feasible in the slack basis, and
 *             runs the dual rule until no rhs is below -eps_r (LP_INFEASIBLE
 *             when a violated row has no entering column); Phase 2 sets the
 *             objective row to z_j = -c_j + sum_i c_B(i) T[i][j] (c_j = 0 for
 *             slacks, the rhs column included), summed over the rows in
 *             increasing order with one fma per row whose basic variable is
 *             structural, restarts the Bland count and runs the primal rule.
 *             Pivots are counted and traced across both phases.  lp_solve
 *             waits for Phase 1 to end before it launches Phase 2.
 *
 * FP32 mode (LP_FP32_REINV; not in the paper): the tableau is FP32, which
 * halves the bytes of the rank-1 update.  Every reinv_k pivots and at
 * termination the library reinverts in FP64 from the original data: for the
 * current basis B it computes x_B = B^-1 b, the duals and the objective row
 * (c_B' B^-1 [A I] - [c 0]) and the objective, rounds them into the FP32
 * tableau's rhs column and objective row, and reports the FP64 values as the
 * solution.  An FP32 optimum is accepted only when these FP64 values are
 * primal and dual feasible within the FP64 tolerances; otherwise pivoting
 * continues (dual simplex from a dual-feasible basis, primal simplex from a
 * primal-feasible one), and LP_NUMERICAL ends a run that does not converge.
 * With lp_options.reinv_body (the default) each reinversion after which the
 * tableau is pivoted again also recomputes its constraint rows B^-1 [A I] in
 * emulated FP64 and rounds them into the FP32 tableau, so pivoting resumes
 * from the correctly rounded tableau of the current basis (an accepted
 * optimum's body, never read again, is left as the FP32 pivots made it).  The FP32 pivot sequence need not equal the
 * FP64 one.
 *
 * Conventions
 *   - Every call returns an lp_err; nothing throws across the ABI.  The
 *     message of the last error of a handle is lp_last_error(handle).
 *   - Solve outcomes (unbounded, iteration limit, ...) are lp_status values,
 *     not errors.
 *   - Pointer arguments may be host or device memory (CUDA unified
 *     addressing tells them apart); the library copies inputs and writes
 *     outputs into caller buffers.  The caller keeps ownership of both.
 *   - The library owns the device memory of a handle (tableau, scratch) and
 *     frees it in lp_destroy.
 *   - A handle is used by one host thread at a time.  Server handles are
 *     thread-safe for submit / poll.
 *   - Matrices are row-major, doubles.
 */
#ifndef GBSIMPLEX_H
#define GBSIMPLEX_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lp_handle lp_handle;

typedef enum {
    LP_OK = 0,
    LP_ERR_INVALID_ARG = 1,      /* bad size, NULL pointer, NaN/Inf input      */
    LP_ERR_OOM = 2,              /* device allocation failed or over budget     */
    LP_ERR_CUDA = 3,             /* a CUDA call failed (message in last_error)  */
    LP_ERR_INFEASIBLE_START = 4, /* LP_MIN_GE with some c_j < 0, or LP_MAX_LE
                                    with some b_i < 0 where no Phase I runs
                                    (FP32 mode, batches, serving, noalloc)     */
    LP_ERR_STATE = 5,            /* call order (solve before load, ...)         */
    LP_ERR_BUSY = 6              /* server: no free slot / budget right now     */
} lp_err;

typedef enum {
    LP_OPTIMAL = 0,
    LP_UNBOUNDED = 1,   /* Sec. 2 Step 3: entering column has no a_iq > eps_p */
    LP_ITER_LIMIT = 2,  /* max_iters pivots made in this call; lp_solve resumes */
    LP_INFEASIBLE = 3,  /* dual simplex: violated row with no T[r][j] < -eps_p */
    LP_NUMERICAL = 4,   /* FP32 mode: FP64 check still fails after reinversions */
    LP_TIMEOUT = 5,     /* a device-side wait exceeded spin_timeout_cycles, or
                           the solve ran past time_limit_s; the tableau is then
                           undefined and lp_solve refuses to resume
                           (LP_ERR_STATE) until the next lp_load               */
    LP_NOT_SOLVED = 6
} lp_status;

typedef enum { LP_MAX_LE = 0, LP_MIN_GE = 1 } lp_sense;
typedef enum { LP_FP64 = 0, LP_FP32_REINV = 1 } lp_precision;

typedef struct {
    int precision;           /* lp_precision                                     */
    int reinv_k;             /* FP32 mode: FP64 reinversion every reinv_k pivots  */
    long long max_iters;     /* pivots per lp_solve call (then LP_ITER_LIMIT)     */
    double eps_d;            /* <= 0: 1e-9 * max(1, max|c|)                       */
    double eps_p;            /* <= 0: 1e-9 * max(1, max|A|)                       */
    double eps_r;            /* <= 0: 1e-9 * max(1, max|b|)                       */
    int bland_after;         /* consecutive zero-ratio pivots before Bland's rule */
    int threads;             /* threads per CTA of the pivot kernel, 0 = auto     */
    long long spin_timeout_cycles; /* device wait limit (SM clock cycles)        */
    void *cuda_stream;       /* cudaStream_t to run on; NULL = library's own      */
    int device;              /* CUDA device ordinal                               */
    int ctas;                /* CTAs of the persistent grid, 0 = auto             */
    long long trace_cap;     /* record (row, column) of the first trace_cap pivots */
    long long group_elems;   /* batched solves: tableau elements per CTA of an LP's
                                group, 0 = 262144 (see lp_solve_batch)            */
    int pipeline;            /* single-LP primal simplex kernel:
                                0 = selection, then update (one launch-wide
                                    grid barrier per pivot);
                                1 = auto (default): 2 below 2^19 tableau
                                    elements ((m+1) x row pitch), else 4; 2
                                    when the second buffer cannot be
                                    allocated;
                                2 = pipelined in place: the next pivot's
                                    selection overlaps this pivot's update, no
                                    grid barrier;
                                3 = pipelined, double-buffered tableau (twice
                                    the memory), a grid barrier per pivot;
                                4 = double-buffered, two pivots per pass over
                                    the tableau (half the tableau traffic per
                                    pivot), no grid barrier between passes;
                                    from m > 4 x 32 x selection warps on, each
                                    CTA forms the new pivot columns on its own
                                    rows and the ratio test is distributed;
                                5 = as 4, the ratio test always distributed.
                                The dual rule (LP_MIN_GE, and FP32 recovery)
                                always runs double-buffered: one pivot per pass
                                for 2 and 3, two for 1, 4 and 5.
                                Same pivots and bits in every mode.              */
    long long solo_elems;    /* servers: an LP of at least this many tableau
                                elements ((m+1) x row pitch) runs alone, as
                                lp_load + lp_solve would run it (the kernels
                                `pipeline` picks; FP32: with its reinversions),
                                once it reaches the head of the queue and the
                                LPs ahead of it are done; 0 = 2^24, < 0 =
                                never.  Ignored elsewhere.                      */
    double time_limit_s;     /* single-LP solves: wall-clock limit in seconds of
                                one lp_solve call (or of lp_solve_async and the
                                wait that completes it), 0 = none.  Past it the
                                host raises an abort word in mapped host memory
                                that every pivot kernel reads once per pass; the
                                kernel stops within a pass and the solve ends in
                                LP_TIMEOUT.  Ignored by batches, servers and
                                lp_solve_noalloc.                               */
    int reinv_body;          /* FP32 mode, single LPs through lp_solve (not the
                                servers, whose HBM budget has no room for the
                                products' workspace): 1 (default) = every reinversion
                                after which the tableau is pivoted again (the
                                periodic ones, one that sends an FP32 optimum
                                back to pivoting, and one that ends a call at
                                the iteration limit) also recomputes the
                                tableau's constraint rows B^-1 [A I] from the
                                original FP64 data, with
                                emulated-FP64 products on the tensor cores (see
                                lp_dgemm_emulated), so the rounding error of the
                                FP32 body does not build up; 0 = only the rhs,
                                the duals and the objective row.  Batches do
                                the latter.                                     */
    int zero_skip;           /* two-pivot primal kernel (pipeline 1, 4, 5: the
                                primal rule, FP64 or the FP32 tableau), on
                                tableaus of at least 2^25 elements ((m+1) x row
                                pitch) with m >= n / 4: 1 (default) = each CTA owns a
                                run of the structural columns and one of the
                                slack and rhs columns, and a pass leaves in
                                place the 16-byte column vectors whose entries
                                in both its pivot rows are zeros (the slack
                                columns of rows whose slack is still basic):
                                Step 5 leaves them bit for bit as they are
                                while no constraint row holds a -0 and the
                                pivot columns are finite, which the kernel
                                tracks (where a -0 may be present, from the
                                data, Phase I or FP32 refreshes, a launch
                                first finds the vectors that hold one).  Each
                                vector's rows live in one of the two tableau
                                buffers; the launch ends with one buffer
                                holding all of them.  0 = every vector
                                updated in every pass; 2 = as 1 at any size
                                and shape (slower where the selection chain
                                bounds the pass).  Same pivots and bits in
                                every mode.                                     */
    long long spill_pivots;  /* servers: 0 (default) = an admitted LP keeps its
                                HBM until it ends.  > 0 = an LP idle on the
                                device that has made at least this many pivots
                                since it was last admitted may be spilled when
                                the request at the head of the queue cannot be
                                admitted (no slot, not enough of the budget,
                                or, for an LP that runs alone, any LP in
                                flight): its tableau and solver state are
                                copied to pinned host memory, its HBM and slot
                                are returned, and it goes to the back of the
                                queue; readmitted, it pivots on from where it
                                stopped, bit for bit as if never spilled.  Idle
                                LPs: those of the FP32 server between its
                                rounds, and an FP64 LP that runs alone
                                (solo_elems), which pivots spill_pivots at a
                                time and is spilled at the end of a slice when
                                any request is waiting.  The LPs of the FP64
                                lanes and of the FP64 server kernel, and FP32
                                LPs that run alone (whose reinversion schedule
                                restarts with each call), run to their end.
                                Ignored elsewhere.                              */
    int lanes;               /* FP64 servers: L in 1..16 (default 3) = L lanes,
                                each solving one LP at a time as lp_load +
                                lp_solve + lp_result would (the kernels
                                `pipeline` picks) on SMs / L CTAs and a 1 / L
                                slice of the budget, the lanes' kernels sharing
                                the GPU; an LP a slice cannot hold runs alone
                                like one of solo_elems elements.  0 = the LPs
                                below solo_elems run in the persistent server
                                kernel instead, each on a group of CTAs with
                                the one-pivot code.  Same bits either way.
                                Ignored elsewhere.                              */
} lp_options;

/* Fill *opt with the defaults: FP64, reinv_k 50, max_iters 1e12, tolerances
 * by formula, bland_after 32, auto launch shape, spin timeout 4e9 cycles,
 * library stream, device 0, no trace, pipelined primal kernel, no wall-clock
 * limit, body refresh on, vectors left in place from 2^25 elements, no
 * spilling, three FP64 server lanes. */
void lp_options_default(lp_options *opt);

/* Create a handle on opt->device (opt may be NULL for the defaults).
 * *out receives the handle, or NULL on error. */
lp_err lp_create(lp_handle **out, const lp_options *opt);

/* Copy one LP into the handle and build its initial tableau (Sec. 2 Step 1:
 * rows [A | I | b], objective row [-c | 0 | 0]; for LP_MIN_GE rows
 * [-A | I | -b] and objective row [c | 0 | 0]).  A is m x n row-major, b has
 * m entries, c has n entries; each may be host or device memory.  m, n >= 1.
 * Replaces any LP loaded before.  LP_MAX_LE with some b_i < 0 is taken in
 * FP64 mode, with Phase I (the header's top).  Errors: LP_ERR_INVALID_ARG
 * (size, NULL, non-finite value), LP_ERR_INFEASIBLE_START (LP_MIN_GE with
 * some c_j < 0; LP_MAX_LE with some b_i < 0 in FP32 mode), LP_ERR_OOM,
 * LP_ERR_CUDA. */
lp_err lp_load(lp_handle *h, int m, int n, const double *A, const double *b,
               const double *c, lp_sense sense);

/* Pivot until optimal, unbounded / infeasible, or max_iters pivots in this
 * call; blocking.  After LP_ITER_LIMIT another call continues from the same
 * tableau.  With opt->time_limit_s > 0 the call ends in LP_TIMEOUT once that
 * much wall time has passed.  Errors: LP_ERR_STATE (nothing loaded, or the
 * last solve ended in LP_TIMEOUT), LP_ERR_CUDA. */
lp_err lp_solve(lp_handle *h);

/* Enqueue the same work on the handle's stream and return without waiting;
 * lp_result (or a stream synchronisation) completes it.  In FP32 mode the
 * host steers the reinversions, so this call waits like lp_solve. */
lp_err lp_solve_async(lp_handle *h);

/* Read the result of the last solve (waits for the handle's stream).
 * x (n entries): primal values, x_j = rhs of the row where j is basic, else 0.
 * y (m entries): dual values, the objective-row entries of the slack columns.
 * obj: c'x.  Any output pointer may be NULL; x, y may be host or device. */
lp_err lp_result(lp_handle *h, double *x, double *y, double *obj,
                 lp_status *status, long long *iters);

/* Diagnostics for tests: the (row, column) of pivots 0..cap-1 of this load
 * (count = pivots recorded), the basic variable of each row, and the
 * (m+1) x (n+m+1) tableau converted to FP64 (host or device buffer). */
lp_err lp_get_trace(lp_handle *h, int *rows, int *cols, long long cap, long long *count);
lp_err lp_get_basis(lp_handle *h, int *basis);
lp_err lp_get_tableau(lp_handle *h, double *T);

/* Device time in milliseconds of the pivot kernel of the last solve, from
 * CUDA events recorded around its launch on the handle's stream (waits for
 * the stream).  *launches receives the number of pivot-kernel launches of
 * that solve (1 in FP64 mode; one per reinversion period in FP32 mode, whose
 * time is summed over them). */
lp_err lp_kernel_time(lp_handle *h, double *ms, int *launches);

/* Batched solve of `count` independent LPs in one persistent launch (the
 * paper solves one LP at a time; batching many uneven LPs is a library
 * service).  LP k is m[k] x n[k] with inputs A[k] (row-major), b[k], c[k]
 * (all host or all device memory) and form sense[k] (NULL: all LP_MAX_LE).
 * Each LP is pivoted by a group of CTAs sized to its tableau
 * (opt->group_elems elements per CTA); CTAs take (LP, rank) work items from a
 * queue, largest LPs first.  Per-LP arithmetic is the single-LP path's, so
 * each result equals solving that LP alone bit for bit.  Outputs per LP:
 * obj[k], status[k], iters[k] and, when x / y and x[k] / y[k] are non-NULL,
 * the primal and dual vectors (host memory).  With opt->precision ==
 * LP_FP32_REINV the tableaus are FP32 and every LP is reinverted in FP64
 * (batched) every reinv_k pivots and at termination, as in the single-LP FP32
 * mode (b >= 0 and c >= 0 required); each result then equals that LP's solo
 * FP32 solve.  opt->threads caps the CTA size at 512; device memory is pooled
 * per device between calls.
 * Blocking.  Errors as lp_load (the message names the LP), in
 * lp_last_error(NULL). */
lp_err lp_solve_batch(int count, const int *m, const int *n, const double *const *A,
                      const double *const *b, const double *const *c, const int *sense,
                      const lp_options *opt, double *obj, lp_status *status, long long *iters,
                      double *const *x, double *const *y);

/* Autotuner for lp_solve_batch: times every candidate launch shape
 * (group_elems in {16K, 64K, 256K, 1M} x threads in {256, 512}) on this
 * batch, best of two solves each, and returns in *best a copy of *opt (NULL:
 * defaults) with the fastest group_elems and threads.  With a non-NULL
 * cache_path the choice is looked up in / appended to that text file, keyed
 * by the batch size and a hash of its sorted shapes. */
lp_err lp_batch_autotune(int count, const int *m, const int *n, const double *const *A,
                         const double *const *b, const double *const *c, const int *sense,
                         const lp_options *opt, const char *cache_path, lp_options *best);

/* Serving with continuous batching (a library service; the paper solves one
 * LP at a time).  A server owns an HBM budget (one arena) and takes requests
 * in arrival order as memory (and, for its kernel, slots) free up.  FP64: by
 * default (opt->lanes) a few lanes each solve one LP at a time as lp_load +
 * lp_solve + lp_result would, on a share of the SMs and a slice of the
 * budget, so the LPs' kernels overlap on the GPU; with opt->lanes 0 a
 * persistent kernel builds, pivots and reads off the admitted LPs (up to
 * max_slots in flight), taking new ones while others run, each on a group of
 * CTAs with the single-LP pivot code.  Either way the result equals solving
 * the LP alone, bit for bit.  An LP of at least opt->solo_elems tableau
 * elements instead runs alone, as lp_load + lp_solve run it, once the LPs
 * ahead of it are done (its buffers come from the same arena).  Inputs are
 * staged in pinned host memory at submit (a pool of reused buffers of up to
 * 8 GiB in all, pageable memory beyond it, freed by lp_server_destroy).
 * m, n <= 4096; inputs and outputs in host memory.
 * With opt->precision == LP_FP32_REINV the tableaus are FP32 and the server
 * works in rounds: one batched launch in which every admitted LP pivots up
 * to reinv_k times, then each LP's FP64 reinversion and the decisions of the
 * FP32 mode (results: the FP64 x, y and objective of the last reinversion);
 * requests are admitted between rounds and pivot in the same launches as the
 * LPs already there.  An LP's rounds do not depend on the others, so its
 * result is the same alone and in the mix, bit for bit.  The FP32 server,
 * like the FP32 mode, needs b >= 0 (max form) and c >= 0 (min form).
 * submit copies the inputs and returns a ticket at once; poll / wait return
 * the result and the submit-to-completion latency in milliseconds (wait
 * returns LP_ERR_BUSY on timeout).  A request whose inputs fail the checks of
 * lp_load completes with that error.  create / destroy are not thread-safe;
 * submit, poll, wait and stats may be called from any thread. */
typedef struct lp_server lp_server;
lp_err lp_server_create(lp_server **out, const lp_options *opt, size_t hbm_budget_bytes,
                        int max_slots);
lp_err lp_server_submit(lp_server *srv, int m, int n, const double *A, const double *b,
                        const double *c, lp_sense sense, unsigned long long *ticket);
lp_err lp_server_poll(lp_server *srv, unsigned long long ticket, int *done, double *x, double *y,
                      double *obj, lp_status *status, long long *iters, double *latency_ms);
lp_err lp_server_wait(lp_server *srv, unsigned long long ticket, double timeout_s, double *x,
                      double *y, double *obj, lp_status *status, long long *iters,
                      double *latency_ms);
/* Requests completed, kernel launches so far, HBM bytes in use, requests
 * waiting for admission. */
lp_err lp_server_stats(lp_server *srv, long long *completed, long long *launches,
                       size_t *hbm_used, int *queued);
/* Spilling (lp_options.spill_pivots): LPs spilled to host memory and
 * readmitted so far, and the pinned host bytes the server holds for spills
 * (buffers are reused; freed by lp_server_destroy).  NULL outputs skipped. */
lp_err lp_server_spill_stats(lp_server *srv, long long *spills, long long *restores,
                             size_t *host_bytes);
/* Finishes the requests in flight, then frees everything.  NULL allowed. */
void lp_server_destroy(lp_server *srv);

/* Figures of the last lp_solve_batch in this process: device time of the
 * batched pivot kernel, total pivots, CTAs launched, CTA size and the largest
 * group. */
lp_err lp_batch_stats(double *kernel_ms, long long *pivots, int *ctas, int *threads,
                      int *max_group);

/* Allocation-free solve (the paper has no counterpart; this is a library
 * service).  Solves one FP64 LP like lp_create + lp_load + lp_solve +
 * lp_result + lp_destroy, but allocates no device or pinned memory: every
 * buffer it needs lives in one fixed 64 MiB device array that the library
 * reserves on each GPU it is loaded on, for the life of the process.  It is
 * for callers that cannot call cudaMalloc when they solve -- code handed a
 * fixed memory budget up front, plug-ins inside a host process that owns the
 * device allocator, loops that must not pay an allocation's latency.
 *   - A (m x n, row-major), b, c: host or device memory; x (n), y (m): host or
 *     device memory or NULL; obj, status, iters: host pointers or NULL.
 *   - opt: NULL for the defaults; FP64 only, opt->trace_cap, opt->pipeline
 *     and opt->time_limit_s are ignored, runs on opt->cuda_stream (NULL: the
 *     legacy default stream) and opt->device; the caller's current device is
 *     restored on return.
 *   - It always runs the one-pivot in-place kernel (pipeline 0: selection,
 *     then the update, one grid barrier per pivot), whose results are bit for
 *     bit those of the other kernels; the pipelined kernels need a second
 *     tableau and more record space than the array holds.
 *   - Blocking: returns after the results are written.
 *   - LPs whose working memory exceeds 64 MiB (about 1500 x 1500) are
 *     rejected with LP_ERR_INVALID_ARG before any GPU work.
 *   - The array is shared by all calls; each call rebuilds or clears what it
 *     uses.  Calls in one process are serialised by a lock; work from it that
 *     overlapped on the GPU (two processes sharing a context) would race.
 *   - The first call on a device looks up the array's device address; make
 *     it before any CUDA stream capture.
 * Errors as lp_load / lp_solve; the message is lp_last_error(NULL). */
lp_err lp_solve_noalloc(int m, int n, const double *A, const double *b, const double *c,
                        lp_sense sense, const lp_options *opt, double *x, double *y,
                        double *obj, lp_status *status, long long *iters);

/* Constraint-row entries the two-pivot primal kernel updated (*updated,
 * each read, updated and written) and left in place (*in_place, see
 * lp_options.zero_skip), in 16-byte vectors times pivots, summed over the
 * solves since lp_load (the objective row, always updated, not counted).
 * Both are 0 for the other kernels.  Either output may be NULL. */
lp_err lp_update_counts(lp_handle *h, long long *updated, long long *in_place);

/* Reinversions of the last FP32 solve, their device time in milliseconds,
 * and the part of it spent recomputing the tableau body (0 with reinv_body
 * off).  Any output may be NULL. */
lp_err lp_fp32_stats(lp_handle *h, int *reinversions, double *reinv_ms, double *body_ms);

/* Emulated-FP64 matrix product on the tensor cores (the paper has no
 * counterpart; it is the engine of the FP32 mode's body refresh):
 * C = A B for FP64 A (M x K, row-major, row pitch lda >= K), B (K x N,
 * row-major, ldb >= N) and C (M x N, row-major, ldc >= N), all device memory.
 * Each row of A and each column of B is scaled by a power of two and split
 * into seven signed 7-bit digits held exactly in bf16; the 28 digit products
 * that carry the leading 49 bits are summed exactly in FP32 on the tensor
 * cores (tcgen05, operands staged by TMA) and combined into FP64.  The error
 * of C_ij is below about K 2^-48 max_k|A_ik| max_k|B_kj| (FP64 itself: K
 * 2^-53 sum_k |A_ik B_kj|); integer data whose products and sums are exact in
 * FP64 and that need at most 14 bits per row or column of scaled magnitude
 * give exact results.  opt: NULL for the defaults; uses opt->device,
 * opt->cuda_stream and opt->spin_timeout_cycles.  Its workspace (about
 * 14 (M + N) K bytes of digit planes) is kept per device between calls, grown
 * when a larger product needs it and held until the process exits; calls are
 * serialised by a lock.  Blocking.  Errors:
 * LP_ERR_INVALID_ARG (sizes, NULL or host pointers), LP_ERR_CUDA (a CUDA call
 * failed or a device wait ran out); the message is lp_last_error(NULL). */
lp_err lp_dgemm_emulated(int M, int N, int K, const double *A, long long lda, const double *B,
                         long long ldb, double *C, long long ldc, const lp_options *opt);
/* The tensor-core MMA instructions (tcgen05.mma kind::f16, 128 x 64 x 16 bf16,
 * 2 x 128 x 64 x 16 flops each) the last lp_dgemm_emulated in this process
 * issued: the digit products it ran, which depend on the data (digit planes
 * that are zero over a whole 128-row or 64-column block are skipped).  0 before
 * the first call or after a failed one. */
lp_err lp_dgemm_stats(long long *tensor_mmas);

/* Free the handle and its device memory.  NULL is allowed. */
void lp_destroy(lp_handle *h);

/* Message of the last error on h ("" if none); h may be NULL for errors of
 * lp_create and the batch call. */
const char *lp_last_error(const lp_handle *h);

/* Library version string. */
const char *lp_version(void);

/* sizeof(lp_options) as compiled into the library, for bindings that lay the
 * struct out themselves. */
size_t lp_options_size(void);

#ifdef __cplusplus
}
#endif

#endif /* GBSIMPLEX_H */
