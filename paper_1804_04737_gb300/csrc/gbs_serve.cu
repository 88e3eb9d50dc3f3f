// Serving engine (lp_server_*): continuous batching of LP requests.
//
// Host side, one engine thread per server:
//   admission   requests wait in FIFO order until a slot and enough of the
//               HBM budget are free; the engine copies their inputs to the
//               device on a copy stream (overlapping the running kernel),
//               writes the slot descriptor and appends the slot to the ring;
//   completion  slots the kernel marked done have their results copied back,
//               their memory returned to the budget and their ticket
//               completed with submit-to-done latency;
//   the kernel  is (re)launched whenever requests are waiting and the last
//               launch has ended (it ends by itself after an idle period).
// Device memory for tableaus comes from one arena of the budget's size,
// managed by a first-fit allocator with coalescing.

#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gbs_internal.h"
#include "gbsimplex.h"

using namespace gbs;

namespace {

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing of free neighbours.
class Arena {
  public:
    void reset(size_t size) {
        free_.clear();
        free_[0] = size;
        size_ = size;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t *off) {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up256(bytes);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }
    size_t size() const { return size_; }

  private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0, used_ = 0;
};

enum TicketState { QUEUED, ADMITTED, DONE };

struct Request {
    int m = 0, n = 0, sense = 0;
    // A, b, c packed (nin doubles): in a pinned buffer of the server's pool
    // (class pin_cls) until the admission copy to the device is done, or in
    // pageable memory when the pool had none to give
    size_t nin = 0;
    double *pin = nullptr;
    int pin_cls = -1;
    std::vector<double> in;
    const double *input() const { return pin ? pin : in.data(); }
    TicketState state = QUEUED;
    int slot = -1;
    size_t off = 0, bytes = 0;
    int group = 1, strip = 0;
    bool solo_oom = false;  // too large to run alone in the arena: served by the kernel
    bool alone = false;     // lanes: too large for a lane's slice of the arena, runs alone
    // results
    std::vector<double> x, y;
    double obj = 0.0;
    int status = LP_NOT_SOLVED;
    long long iters = 0;
    lp_err err = LP_OK;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    // spilled to pinned host memory (lp_options.spill_pivots): FP32 rounds,
    // the slot's bytes and the engine's state of the LP; an LP run alone,
    // the bytes of its handle's range of the arena (the handle keeps the
    // host-side state)
    bool spilled = false;
    unsigned char *host = nullptr;
    size_t host_cap = 0;            // bytes of the pinned buffer
    size_t host_used = 0;           // bytes copied into it
    long long resident_from = 0;    // pivots made when last (re)admitted
    LpDesc d32{};
    int rule32 = 0, failed32 = 0;
    long long remaining32 = 0, guard32 = 0;
    lp_handle *solo_h = nullptr;
};

}  // namespace

struct lp_server {
    lp_options opt;
    int device = 0, sms = 0, threads = 512, ctas = 0, workers = 0;
    size_t smem = 0;
    int max_slots = 0;
    static constexpr int kMaxDim = 4096;
    cudaStream_t kstream = nullptr, cstream = nullptr;
    unsigned char *arena_dev = nullptr;
    Arena arena;
    ServeSlot *d_slots = nullptr;
    ServeCtl *d_ctl = nullptr;
    ServeRing *h_ring = nullptr, *d_ring = nullptr;
    std::vector<int> free_slots;
    std::vector<unsigned long long> slot_ticket;
    std::mutex mu;
    std::condition_variable cv;
    std::unordered_map<unsigned long long, Request> reqs;
    std::deque<unsigned long long> queue;
    unsigned long long next_ticket = 1;
    std::thread engine;
    std::atomic<bool> stop{false};
    bool kernel_running = false;
    cudaEvent_t kdone = nullptr;
    long long launches = 0, completed = 0;
    // an LP of at least solo_elems tableau elements is solved alone, on a
    // library handle whose buffers are the arena, by the single-LP kernels
    // (two pivots per pass over the tableau on every SM; in FP32 mode with its
    // FP64 reinversions), once the LPs admitted before it are done (FP64: the
    // persistent kernel has finished them and exited; FP32: no LP is in a round)
    long long solo_elems = -1;
    lp_handle *solo = nullptr;
    lp_err fatal = LP_OK;
    char fatal_msg[256] = {0};
    // FP32 tableaus with FP64 reinversion (precision LP_FP32_REINV): a round
    // engine instead of the persistent kernel.  Each round is one batched
    // launch in which every admitted LP pivots up to reinv_k times, then the
    // FP64 reinversion and decision of each LP; requests are admitted
    // between rounds, so new LPs pivot in the same launches as older ones.
    bool fp32 = false;
    LpDesc *d_desc32 = nullptr, *h_desc32 = nullptr;  // one per slot (host copy pinned)
    int2 *d_items = nullptr, *h_items = nullptr;        // a round's work items
    unsigned *d_queue = nullptr;
    int ctas32 = 0;
    size_t smem32 = 0;
    std::vector<int> active;  // slots being pivoted
    std::vector<int> rule, failed;
    std::vector<long long> remaining, guard, before;
    ReinvPool *rp = nullptr;
    BatchReinv ws32;
    // spilling (lp_options.spill_pivots): pinned host buffers not in use, by
    // size, every pinned buffer allocated, and the counts
    long long spill_pivots = 0;
    // FP64 lanes (lp_options.lanes > 0) instead of the persistent kernel: the
    // lane threads, their handles' CTA count and arena slice, the lanes that
    // are solving an LP; alone_wait: an LP that runs alone is at the head of
    // the queue (lanes start no new LP), alone_busy: it is running
    int lanes = 0, lane_ctas = 0;
    size_t lane_bytes = 0;
    std::vector<std::thread> lane_threads;
    int busy_lanes = 0;
    bool alone_wait = false, alone_busy = false;
    // pinned buffers for request inputs, by size class (2^k bytes), and
    // every one allocated (pin_mu: submit runs on the callers' threads)
    std::mutex pin_mu;
    std::vector<std::vector<double *>> pin_free;
    std::vector<void *> pin_all;
    size_t pin_total = 0;
    std::multimap<size_t, unsigned char *> host_free;
    std::vector<std::pair<unsigned char *, size_t>> host_all;
    size_t host_total = 0;
    long long spills = 0, restores = 0;
};

namespace {

lp_err sfail(lp_err code, const char *fmt, ...) {
    char msg[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof msg, fmt, ap);
    va_end(ap);
    set_last_error_global(msg);
    return code;
}

struct SlotLayout {
    size_t T, in, basis, part, bar, out, stats, total;
};

SlotLayout slot_layout(int m, int n, long long P, int G, size_t esz = sizeof(double)) {
    SlotLayout L;
    size_t off = 0;
    auto take = [&](size_t b) { const size_t at = off; off += up256(b); return at; };
    L.T = take((size_t)(m + 1) * (size_t)P * esz);
    L.in = take(((size_t)m * n + m + n) * sizeof(double));
    L.basis = take((size_t)m * sizeof(int));
    L.part = take(2 * (size_t)G * sizeof(Cand));
    L.bar = take(512);
    L.out = take(((size_t)n + m + 1) * sizeof(double));
    L.stats = take(sizeof(InputStats));
    L.total = off;
    return L;
}

void group_shape(const lp_server *sv, int m, int n, int *G, int *W) {
    const long long M = m + 1, P = pitch_for(n + m + 1);
    const long long ge = sv->opt.group_elems > 0 ? sv->opt.group_elems : 262144;
    const long long gmin = (P + (long long)sv->threads * 2 - 1) / ((long long)sv->threads * 2);
    long long g = (M * P + ge - 1) / ge;
    g = std::min<long long>(g, std::min<long long>(sv->workers, P / 4));
    g = std::max<long long>(g, gmin);
    long long w = (P + g - 1) / g;
    w = (w + 3) / 4 * 4;
    *W = (int)w;
    *G = (int)((P + w - 1) / w);
}

// The FP32 engine's group of CTAs and strip width for one LP (FP32 vectors of
// four, strips of whole 32-byte sectors), as the FP32 batch path sizes them.
void group_shape32(const lp_server *sv, int m, int n, int *G, int *W) {
    const long long M = m + 1, P = pitch_for(n + m + 1);
    const long long ge = sv->opt.group_elems > 0 ? sv->opt.group_elems : 262144;
    const long long gmin = (P + (long long)sv->threads * 4 - 1) / ((long long)sv->threads * 4);
    long long g = (M * P + ge - 1) / ge;
    g = std::min<long long>(g, std::min<long long>(sv->ctas32, P / 8));
    g = std::max<long long>(g, gmin);
    long long w = (P + g - 1) / g;
    w = (w + 7) / 8 * 8;
    *W = (int)w;
    *G = (int)((P + w - 1) / w);
}

bool is_solo(const lp_server *sv, const Request &r) {
    return r.alone || (sv->solo_elems >= 0 && !r.solo_oom &&
                       (long long)(r.m + 1) * pitch_for(r.n + r.m + 1) >= sv->solo_elems);
}

// A max-form request with some b_i < 0 (and every input finite; lp_load
// reports a non-finite one): the server has no Phase I, so it is rejected
// with LP_ERR_INFEASIBLE_START, as the server kernel rejects it.
bool needs_phase1(const Request &r) {
    if (r.sense != LP_MAX_LE) return false;
    const double *A = r.input(), *b = A + (size_t)r.m * r.n;
    bool neg = false;
    for (int i = 0; i < r.m; ++i) neg |= b[i] < 0.0;
    if (!neg) return false;
    for (size_t k = 0; k < r.nin; ++k)
        if (!isfinite(A[k])) return false;
    return true;
}

// A server-wide failure: every waiting call returns `code` from now on.
void set_fatal(lp_server *sv, lp_err code, const char *what, cudaError_t e) {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->fatal = code;
    snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "%s: %s", what, cudaGetErrorString(e));
    sv->cv.notify_all();
}

// A pinned host buffer of at least `bytes` for a spill: the smallest free
// one of at most twice the size, else a new one (nullptr when the host
// cannot pin more; the LP then stays).
unsigned char *host_take(lp_server *sv, size_t bytes, size_t *cap) {
    auto it = sv->host_free.lower_bound(bytes);
    if (it != sv->host_free.end() && it->first / 2 <= bytes) {
        unsigned char *p = it->second;
        *cap = it->first;
        sv->host_free.erase(it);
        return p;
    }
    void *p = nullptr;
    if (cudaHostAlloc(&p, std::max<size_t>(bytes, 1), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    sv->host_all.push_back({static_cast<unsigned char *>(p), bytes});
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->host_total += bytes;
    *cap = bytes;
    return static_cast<unsigned char *>(p);
}

void host_give(lp_server *sv, unsigned char *p, size_t cap) { sv->host_free.emplace(cap, p); }

// Pinned host memory for a request's inputs, so that admission copies them to
// the device by DMA at the link's rate instead of through the driver's
// staging of pageable memory (measured: 0.68 ms of each lp_load's 1.4 ms on
// the serving stream's LPs, 7.5 MB of inputs on average).  Buffers of 2^k
// bytes, reused; at most kPinInputCap bytes in all, beyond which requests
// keep their inputs in pageable memory.
constexpr size_t kPinInputCap = 8ull << 30;

double *pin_take(lp_server *sv, size_t bytes, int *cls) {
    int k = 12;
    while (((size_t)1 << k) < bytes) ++k;
    std::lock_guard<std::mutex> lk(sv->pin_mu);
    if ((int)sv->pin_free.size() <= k) sv->pin_free.resize(k + 1);
    if (!sv->pin_free[k].empty()) {
        double *p = sv->pin_free[k].back();
        sv->pin_free[k].pop_back();
        *cls = k;
        return p;
    }
    if (sv->pin_total + ((size_t)1 << k) > kPinInputCap) return nullptr;
    DeviceRestore restore_;
    void *p = nullptr;
    if (cudaSetDevice(sv->device) != cudaSuccess ||
        cudaHostAlloc(&p, (size_t)1 << k, cudaHostAllocPortable) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    sv->pin_all.push_back(p);
    sv->pin_total += (size_t)1 << k;
    *cls = k;
    return static_cast<double *>(p);
}

// The request's pinned inputs back to the pool (their copy to the device is
// complete, or they are not needed any more).
void pin_give(lp_server *sv, Request &r) {
    if (!r.pin) return;
    std::lock_guard<std::mutex> lk(sv->pin_mu);
    sv->pin_free[r.pin_cls].push_back(r.pin);
    r.pin = nullptr;
    r.pin_cls = -1;
}

// Copy results of finished slots back and release their resources.
bool engine_complete(lp_server *sv) {
    std::vector<int> fin;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (int s = 0; s < sv->max_slots; ++s)
            if (sv->slot_ticket[s] && *(volatile int *)&sv->h_ring->done[s] == 1) fin.push_back(s);
    }
    if (fin.empty()) return false;
    std::atomic_thread_fence(std::memory_order_acquire);
    for (int s : fin) {
        Request *r;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r = &sv->reqs[sv->slot_ticket[s]];
        }
        const long long P = pitch_for(r->n + r->m + 1);
        const SlotLayout L = slot_layout(r->m, r->n, P, r->group);
        LpDesc d;
        r->x.resize(r->n);
        r->y.resize(r->m);
        const double *out = reinterpret_cast<const double *>(sv->arena_dev + r->off + L.out);
        cudaMemcpyAsync(&d, &sv->d_slots[s].d, sizeof d, cudaMemcpyDeviceToHost, sv->cstream);
        cudaMemcpyAsync(r->x.data(), out, sizeof(double) * r->n, cudaMemcpyDeviceToHost, sv->cstream);
        cudaMemcpyAsync(r->y.data(), out + r->n, sizeof(double) * r->m, cudaMemcpyDeviceToHost,
                        sv->cstream);
        cudaMemcpyAsync(&r->obj, out + r->n + r->m, sizeof(double), cudaMemcpyDeviceToHost,
                        sv->cstream);
        cudaStreamSynchronize(sv->cstream);
        std::lock_guard<std::mutex> lk(sv->mu);
        r->iters = d.iters;
        if (d.status == -2) { r->err = LP_ERR_INVALID_ARG; r->status = LP_NOT_SOLVED; }
        else if (d.status == -3) { r->err = LP_ERR_INFEASIBLE_START; r->status = LP_NOT_SOLVED; }
        else r->status = d.status;
        r->state = DONE;
        r->t_done = now_ms();
        sv->arena.release(r->off, r->bytes);
        sv->slot_ticket[s] = 0;
        sv->free_slots.push_back(s);
        *(volatile int *)&sv->h_ring->done[s] = 0;
        ++sv->completed;
    }
    sv->cv.notify_all();
    return true;
}

// Move waiting requests into free slots while the budget allows (FIFO).
bool engine_admit(lp_server *sv) {
    struct Adm { int s; unsigned long long t; Request *r; };
    std::vector<Adm> adm;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        while (!sv->queue.empty() && !sv->free_slots.empty()) {
            const unsigned long long t = sv->queue.front();
            Request &r = sv->reqs[t];
            if (is_solo(sv, r)) break;
            group_shape(sv, r.m, r.n, &r.group, &r.strip);
            const SlotLayout L = slot_layout(r.m, r.n, pitch_for(r.n + r.m + 1), r.group);
            size_t off;
            if (!sv->arena.alloc(L.total, &off)) break;
            r.off = off;
            r.bytes = L.total;
            r.slot = sv->free_slots.back();
            sv->free_slots.pop_back();
            sv->slot_ticket[r.slot] = t;
            r.state = ADMITTED;
            r.t_admit = now_ms();
            sv->queue.pop_front();
            adm.push_back({r.slot, t, &r});
        }
    }
    if (adm.empty()) return false;
    std::vector<ServeSlot> hs(adm.size());
    for (size_t k = 0; k < adm.size(); ++k) {
        Request &r = *adm[k].r;
        const int m = r.m, n = r.n;
        const long long P = pitch_for(n + m + 1);
        const SlotLayout L = slot_layout(m, n, P, r.group);
        unsigned char *base = sv->arena_dev + r.off;
        cudaMemcpyAsync(base + L.in, r.input(), r.nin * sizeof(double), cudaMemcpyHostToDevice,
                        sv->cstream);
        cudaMemsetAsync(base + L.bar, 0, 512, sv->cstream);
        cudaMemsetAsync(base + L.stats, 0, sizeof(InputStats), sv->cstream);
        ServeSlot &S = hs[k];
        memset(&S, 0, sizeof S);
        LpDesc &d = S.d;
        d.T = base + L.T;
        d.basis = reinterpret_cast<int *>(base + L.basis);
        d.part_sel = reinterpret_cast<Cand *>(base + L.part);
        d.bar = reinterpret_cast<unsigned *>(base + L.bar);
        d.err = reinterpret_cast<int *>(d.bar + 96);
        d.P = P;
        d.m = m;
        d.n = n;
        d.M = m + 1;
        d.N = n + m + 1;
        d.sense = r.sense;
        d.bland_after = sv->opt.bland_after;
        d.status = -1;
        d.last_p = d.last_q = -1;
        d.group = r.group;
        d.strip = r.strip;
        const double *in = reinterpret_cast<const double *>(base + L.in);
        S.A = in;
        S.b = in + (size_t)m * n;
        S.c = S.b + m;
        double *out = reinterpret_cast<double *>(base + L.out);
        S.x = out;
        S.y = out + n;
        S.obj = out + n + m;
        S.stats = reinterpret_cast<InputStats *>(base + L.stats);
        S.opt_eps_d = sv->opt.eps_d;
        S.opt_eps_p = sv->opt.eps_p;
        S.opt_eps_r = sv->opt.eps_r;
        S.budget = sv->opt.max_iters;
        cudaMemcpyAsync(&sv->d_slots[adm[k].s], &S, sizeof S, cudaMemcpyHostToDevice, sv->cstream);
    }
    cudaStreamSynchronize(sv->cstream);
    for (const Adm &a : adm) pin_give(sv, *a.r);
    int tail = *(volatile int *)&sv->h_ring->rq_tail;
    for (const Adm &a : adm) sv->h_ring->rq[tail++ % kServeMaxSlots] = a.s;
    std::atomic_thread_fence(std::memory_order_release);
    *(volatile int *)&sv->h_ring->rq_tail = tail;
    return true;
}

void engine_kernel(lp_server *sv) {
    if (sv->kernel_running && cudaEventQuery(sv->kdone) == cudaSuccess) {
        sv->kernel_running = false;
        int err = 0;
        cudaMemcpy(&err, &sv->d_ctl->err, sizeof err, cudaMemcpyDeviceToHost);
        if (err) {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->fatal = LP_ERR_CUDA;
            snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "server kernel: a device wait timed out");
            sv->cv.notify_all();
        }
    }
    bool pending;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        pending = sv->fatal == LP_OK &&
                  *(volatile int *)&sv->h_ring->rq_head != *(volatile int *)&sv->h_ring->rq_tail;
        for (int s = 0; !pending && s < sv->max_slots; ++s)
            if (sv->slot_ticket[s] && *(volatile int *)&sv->h_ring->done[s] == 0) pending = true;
    }
    if (!pending || sv->kernel_running) return;
    cudaMemsetAsync(sv->d_ctl, 0, sizeof(ServeCtl), sv->kstream);
    const long long idle = 100000000ll;  // ~50 ms of SM clock with no work
    cudaError_t e = launch_server(sv->d_slots, sv->max_slots, sv->d_ctl, sv->d_ring, sv->ctas,
                                  sv->threads, sv->smem, sv->opt.spin_timeout_cycles, idle,
                                  sv->kstream);
    if (e == cudaSuccess) e = cudaEventRecord(sv->kdone, sv->kstream);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->fatal = LP_ERR_CUDA;
        snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "server launch: %s", cudaGetErrorString(e));
        sv->cv.notify_all();
        return;
    }
    sv->kernel_running = true;
    ++sv->launches;
}

// bits of a double (the input statistics hold the bits of max |.|)
double bits_double(unsigned long long b) {
    double v;
    memcpy(&v, &b, sizeof v);
    return v;
}

// ---- FP32 engine ----

// Finish the request in `slot`: its FP64 results (those of the last
// reinversion), its status, and the slot's memory back to the budget.
void finish32(lp_server *sv, int slot, int status, lp_err err) {
    Request *r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r = &sv->reqs[sv->slot_ticket[slot]];
    }
    const LpDesc &d = sv->h_desc32[slot];
    // sized in every case: the results are copied out of these on completion
    r->x.assign(r->n, 0.0);
    r->y.assign(r->m, 0.0);
    if (err == LP_OK) {
        const long long P = pitch_for(r->n + r->m + 1);
        const SlotLayout L = slot_layout(r->m, r->n, P, r->group, sizeof(float));
        const double *out = reinterpret_cast<const double *>(sv->arena_dev + r->off + L.out);
        cudaMemcpyAsync(r->x.data(), out, sizeof(double) * r->n, cudaMemcpyDeviceToHost, sv->kstream);
        cudaMemcpyAsync(r->y.data(), out + r->n, sizeof(double) * r->m, cudaMemcpyDeviceToHost,
                        sv->kstream);
        cudaMemcpyAsync(&r->obj, out + r->n + r->m, sizeof(double), cudaMemcpyDeviceToHost,
                        sv->kstream);
        cudaStreamSynchronize(sv->kstream);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    r->iters = err == LP_OK ? d.iters : 0;
    r->err = err;
    r->status = err == LP_OK ? status : LP_NOT_SOLVED;
    r->state = DONE;
    r->t_done = now_ms();
    sv->arena.release(r->off, r->bytes);
    sv->slot_ticket[slot] = 0;
    sv->free_slots.push_back(slot);
    ++sv->completed;
    sv->cv.notify_all();
}

// Admit waiting requests (FIFO, while a slot and the budget allow): copy the
// inputs, check them, build the FP32 tableau and the slot's descriptor.
bool admit32(lp_server *sv) {
    std::vector<std::pair<int, Request *>> adm;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        while (!sv->queue.empty() && !sv->free_slots.empty()) {
            const unsigned long long t = sv->queue.front();
            Request &r = sv->reqs[t];
            if (is_solo(sv, r)) break;
            if (!r.spilled) group_shape32(sv, r.m, r.n, &r.group, &r.strip);
            const SlotLayout L = slot_layout(r.m, r.n, pitch_for(r.n + r.m + 1), r.group, sizeof(float));
            size_t off;
            if (!sv->arena.alloc(L.total, &off)) break;
            r.off = off;
            r.bytes = L.total;
            r.slot = sv->free_slots.back();
            sv->free_slots.pop_back();
            sv->slot_ticket[r.slot] = t;
            r.state = ADMITTED;
            r.t_admit = now_ms();
            sv->queue.pop_front();
            adm.push_back({r.slot, &r});
        }
    }
    if (adm.empty()) return false;
    cudaStream_t s = sv->kstream;
    std::vector<InputStats> st(adm.size());
    for (size_t k = 0; k < adm.size(); ++k) {
        Request &r = *adm[k].second;
        const SlotLayout L = slot_layout(r.m, r.n, pitch_for(r.n + r.m + 1), r.group, sizeof(float));
        unsigned char *base = sv->arena_dev + r.off;
        if (r.spilled) {  // the slot's bytes as they were spilled
            cudaMemcpyAsync(base, r.host, r.host_used, cudaMemcpyHostToDevice, s);
            continue;
        }
        const double *A = reinterpret_cast<const double *>(base + L.in);
        cudaMemcpyAsync(base + L.in, r.input(), r.nin * sizeof(double), cudaMemcpyHostToDevice, s);
        cudaMemsetAsync(base + L.bar, 0, 512, s);
        launch_inspect(A, A + (size_t)r.m * r.n, A + (size_t)r.m * r.n + r.m, r.m, r.n,
                       reinterpret_cast<InputStats *>(base + L.stats), s);
        cudaMemcpyAsync(&st[k], base + L.stats, sizeof(InputStats), cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        set_fatal(sv, LP_ERR_CUDA, "FP32 admission", ce);
        return true;
    }
    for (auto &a : adm) pin_give(sv, *a.second);
    for (size_t k = 0; k < adm.size(); ++k) {
        const int slot = adm[k].first;
        Request &r = *adm[k].second;
        const int m = r.m, n = r.n;
        const long long P = pitch_for(n + m + 1);
        const SlotLayout L = slot_layout(m, n, P, r.group, sizeof(float));
        unsigned char *base = sv->arena_dev + r.off;
        if (r.spilled) {
            // readmitted: the descriptor's pointers into the slot's new
            // place, the engine's state as it was
            LpDesc d = r.d32;
            d.T = base + L.T;
            d.basis = reinterpret_cast<int *>(base + L.basis);
            d.part_sel = reinterpret_cast<Cand *>(base + L.part);
            d.bar = reinterpret_cast<unsigned *>(base + L.bar);
            d.err = reinterpret_cast<int *>(d.bar + 96);
            sv->h_desc32[slot] = d;
            sv->rule[slot] = r.rule32;
            sv->failed[slot] = r.failed32;
            sv->remaining[slot] = r.remaining32;
            sv->guard[slot] = r.guard32;
            sv->active.push_back(slot);
            host_give(sv, r.host, r.host_cap);
            std::lock_guard<std::mutex> lk(sv->mu);
            r.host = nullptr;
            r.spilled = false;
            r.resident_from = d.iters;
            ++sv->restores;
            continue;
        }
        lp_err err = LP_OK;
        if (st[k].flags & 4) err = LP_ERR_INVALID_ARG;
        else if (r.sense == LP_MAX_LE && (st[k].flags & 1)) err = LP_ERR_INFEASIBLE_START;
        else if (r.sense == LP_MIN_GE && (st[k].flags & 2)) err = LP_ERR_INFEASIBLE_START;
        if (err != LP_OK) {
            finish32(sv, slot, LP_NOT_SOLVED, err);
            continue;
        }
        const double *A = reinterpret_cast<const double *>(base + L.in);
        LpDesc d{};
        d.T = base + L.T;
        d.basis = reinterpret_cast<int *>(base + L.basis);
        d.part_sel = reinterpret_cast<Cand *>(base + L.part);
        d.bar = reinterpret_cast<unsigned *>(base + L.bar);
        d.err = reinterpret_cast<int *>(d.bar + 96);
        d.P = P;
        d.m = m;
        d.n = n;
        d.M = m + 1;
        d.N = n + m + 1;
        d.sense = r.sense;
        d.bland_after = sv->opt.bland_after;
        // the FP32 tableau pivots with the FP64 tolerances (as lp_load's FP32 mode)
        d.eps_d = sv->opt.eps_d > 0 ? sv->opt.eps_d : 1e-9 * std::max(1.0, bits_double(st[k].cmax_bits));
        d.eps_p = sv->opt.eps_p > 0 ? sv->opt.eps_p : 1e-9 * std::max(1.0, bits_double(st[k].amax_bits));
        d.eps_r = sv->opt.eps_r > 0 ? sv->opt.eps_r : 1e-9 * std::max(1.0, bits_double(st[k].bmax_bits));
        d.status = -1;
        d.last_p = d.last_q = -1;
        d.group = r.group;
        d.strip = r.strip;
        launch_build(PREC_FP32, A, A + (size_t)m * n, A + (size_t)m * n + m, m, n, r.sense, d.T, P,
                     d.basis, s);
        sv->h_desc32[slot] = d;
        sv->rule[slot] = r.sense;
        sv->failed[slot] = 0;
        sv->remaining[slot] = sv->opt.max_iters;
        sv->guard[slot] = 20ll * (m + n) + 1000;
        sv->active.push_back(slot);
        r.resident_from = 0;
    }
    return true;
}

// Spill the FP32 LP in `slot`, idle between rounds: the slot's bytes to a
// pinned host buffer, the descriptor and the engine's state of the LP to the
// request; the slot and its HBM are returned and the request goes to the back
// of the queue.  False (the LP stays) when no host buffer can be had.
bool spill32(lp_server *sv, int slot) {
    unsigned long long t;
    Request *r;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        t = sv->slot_ticket[slot];
        r = &sv->reqs[t];
    }
    size_t cap = 0;
    unsigned char *hp = host_take(sv, r->bytes, &cap);
    if (!hp) return false;
    cudaError_t e = cudaMemcpyAsync(hp, sv->arena_dev + r->off, r->bytes, cudaMemcpyDeviceToHost,
                                    sv->kstream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(sv->kstream);
    if (e != cudaSuccess) {
        host_give(sv, hp, cap);
        set_fatal(sv, LP_ERR_CUDA, "FP32 spill", e);
        return false;
    }
    r->d32 = sv->h_desc32[slot];
    r->rule32 = sv->rule[slot];
    r->failed32 = sv->failed[slot];
    r->remaining32 = sv->remaining[slot];
    r->guard32 = sv->guard[slot];
    const auto at = std::find(sv->active.begin(), sv->active.end(), slot);
    if (at != sv->active.end()) sv->active.erase(at);
    std::lock_guard<std::mutex> lk(sv->mu);
    r->host = hp;
    r->host_cap = cap;
    r->host_used = r->bytes;
    r->spilled = true;
    sv->arena.release(r->off, r->bytes);
    sv->slot_ticket[slot] = 0;
    sv->free_slots.push_back(slot);
    r->slot = -1;
    r->state = QUEUED;
    sv->queue.push_back(t);
    ++sv->spills;
    return true;
}

// Between rounds, with spill_pivots > 0: when the request at the head of the
// queue cannot be admitted (no free slot or not enough of the budget), spill
// the LPs in the rounds that have pivoted at least spill_pivots times since
// they were last admitted, longest-running first, until it can; for an LP
// that runs alone (which needs the whole arena) only once every LP in the
// rounds may go.  Nothing is spilled when the eligible LPs could not make
// room.
void evict32(lp_server *sv) {
    if (sv->spill_pivots <= 0 || sv->active.empty()) return;
    std::vector<std::pair<long long, int>> cand;  // (pivots since admission, slot)
    bool solo = false;
    size_t need = 0, freeable = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->fatal != LP_OK || sv->queue.empty()) return;
        for (int slot : sv->active) {
            const Request &r = sv->reqs[sv->slot_ticket[slot]];
            const long long run = sv->h_desc32[slot].iters - r.resident_from;
            if (run >= sv->spill_pivots) {
                cand.push_back({run, slot});
                freeable += up256(r.bytes);
            }
        }
        if (cand.empty()) return;
        Request &h = sv->reqs[sv->queue.front()];
        solo = is_solo(sv, h);
        if (!solo) {
            if (!h.spilled) group_shape32(sv, h.m, h.n, &h.group, &h.strip);
            need = up256(slot_layout(h.m, h.n, pitch_for(h.n + h.m + 1), h.group, sizeof(float)).total);
            if (sv->arena.size() - sv->arena.used() + freeable < need) return;
        }
    }
    std::stable_sort(cand.begin(), cand.end(),
                     [](const std::pair<long long, int> &a, const std::pair<long long, int> &b) {
                         return a.first > b.first;
                     });
    if (solo) {
        if (cand.size() != sv->active.size()) return;
        for (const auto &c : cand)
            if (!spill32(sv, c.second)) return;
        return;
    }
    auto admissible = [&]() {
        std::lock_guard<std::mutex> lk(sv->mu);
        size_t off;
        if (sv->free_slots.empty() || !sv->arena.alloc(need, &off)) return false;
        sv->arena.release(off, need);
        return true;
    };
    for (const auto &c : cand) {
        if (admissible()) return;
        if (!spill32(sv, c.second)) return;
    }
}

// One round: every admitted LP pivots up to reinv_k times in one batched
// FP32 launch, then, LP by LP, the FP64 reinversion of its basis and the
// decisions of the FP32 batch path (accept an FP32 optimum only when the
// FP64 values are primal and dual feasible; otherwise continue with the rule
// whose invariant holds).
void round32(lp_server *sv) {
    cudaStream_t s = sv->kstream;
    std::vector<int> order = sv->active;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return (long long)sv->h_desc32[a].M * sv->h_desc32[a].P >
               (long long)sv->h_desc32[b].M * sv->h_desc32[b].P;
    });
    long long budget = sv->opt.reinv_k;
    int nitems = 0;
    for (int slot : order) {
        LpDesc &d = sv->h_desc32[slot];
        budget = std::min(budget, sv->remaining[slot]);
        for (int r = 0; r < d.group; ++r) sv->h_items[nitems++] = make_int2(slot, r);
        d.sense = sv->rule[slot];
        sv->before[slot] = d.iters;
        cudaMemsetAsync(d.bar, 0, 512, s);
    }
    cudaMemcpyAsync(sv->d_items, sv->h_items, nitems * sizeof(int2), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(sv->d_desc32, sv->h_desc32, sv->max_slots * sizeof(LpDesc),
                    cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(sv->d_queue, 0, sizeof(unsigned), s);
    cudaError_t e = launch_batch(PREC_FP32, sv->d_desc32, sv->d_items, nitems, sv->d_queue,
                                 sv->ctas32, sv->threads, sv->smem32, 1,
                                 sv->opt.spin_timeout_cycles, budget, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sv->h_desc32, sv->d_desc32, sv->max_slots * sizeof(LpDesc),
                            cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->fatal = LP_ERR_CUDA;
        snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "FP32 round: %s", cudaGetErrorString(e));
        sv->cv.notify_all();
        return;
    }
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        ++sv->launches;
    }
    // the FP64 reinversion of every active LP's basis, batched
    std::vector<int> idx;
    std::vector<ReinvJob> jobs;
    for (int slot : sv->active) {
        LpDesc &d = sv->h_desc32[slot];
        Request *r;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            r = &sv->reqs[sv->slot_ticket[slot]];
        }
        const long long made = d.iters - sv->before[slot];
        sv->remaining[slot] -= made;
        sv->guard[slot] -= made;
        if (d.status == LP_TIMEOUT) {
            finish32(sv, slot, LP_TIMEOUT, LP_OK);
            continue;
        }
        const int m = r->m, n = r->n;
        const long long P = pitch_for(n + m + 1);
        const SlotLayout L = slot_layout(m, n, P, r->group, sizeof(float));
        unsigned char *base = sv->arena_dev + r->off;
        const double *A = reinterpret_cast<const double *>(base + L.in), *b = A + (size_t)m * n,
                     *c = b + m;
        double *out = reinterpret_cast<double *>(base + L.out);
        jobs.push_back(ReinvJob{A, b, c, m, n, r->sense, d.basis, d.T, P, out, out + n, out + n + m});
        idx.push_back(slot);
    }
    int badj = -1;
    e = reinvert_many(PREC_FP32, jobs.data(), (int)jobs.size(), sv->ws32, *sv->rp, sv->sms,
                      sv->opt.spin_timeout_cycles, s, &badj);
    if (e != cudaSuccess || badj >= 0) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->fatal = LP_ERR_CUDA;
        snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "FP32 reinversion: %s",
                 e != cudaSuccess ? cudaGetErrorString(e) : "inconsistent basis");
        sv->cv.notify_all();
        return;
    }
    std::vector<int> still;
    for (size_t q = 0; q < idx.size(); ++q) {
        const int slot = idx[q];
        LpDesc &d = sv->h_desc32[slot];
        const int st = d.status;
        const ReinvCheck *chk = sv->ws32.h_chk + q;
        if (chk->singular) {
            finish32(sv, slot, LP_NUMERICAL, LP_OK);
            continue;
        }
        const bool pfeas = key_to_double(chk->rhsmin_key) >= -d.eps_r;
        const bool dfeas = key_to_double(chk->zmin_key) >= -d.eps_d;
        if (st == LP_OPTIMAL) {
            if (pfeas && dfeas) {
                finish32(sv, slot, LP_OPTIMAL, LP_OK);
            } else if ((!pfeas && !dfeas) || ++sv->failed[slot] > 4) {
                finish32(sv, slot, LP_NUMERICAL, LP_OK);
            } else {
                sv->rule[slot] = pfeas ? 0 : 1;
                still.push_back(slot);
            }
            continue;
        }
        if (st == LP_UNBOUNDED || st == LP_INFEASIBLE) {
            finish32(sv, slot, st, LP_OK);
            continue;
        }
        if (sv->remaining[slot] <= 0) {
            finish32(sv, slot, LP_ITER_LIMIT, LP_OK);
            continue;
        }
        if (sv->guard[slot] <= 0) {
            finish32(sv, slot, LP_NUMERICAL, LP_OK);
            continue;
        }
        if (sv->rule[slot] == 0 && !pfeas && dfeas) sv->rule[slot] = 1;
        else if (sv->rule[slot] == 1 && !dfeas && pfeas) sv->rule[slot] = 0;
        still.push_back(slot);
    }
    sv->active.swap(still);
}

bool engine_solo(lp_server *sv);

void engine32_main(lp_server *sv) {
    cudaSetDevice(sv->device);
    while (!sv->stop.load()) {
        bool fatal;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            fatal = sv->fatal != LP_OK;
        }
        if (!fatal) evict32(sv);
        const bool admitted = !fatal && admit32(sv);
        if (!fatal && !sv->active.empty()) {
            round32(sv);
        } else if (!admitted && (fatal || !engine_solo(sv))) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

// A large LP at the head of the queue.  While LPs admitted before it are in
// flight (admission stops at this LP), ask the FP64 persistent kernel to exit
// once they are done, or let the FP32 rounds finish them; then solve the LP on
// the library handle, its buffers carved from the whole (now empty) arena,
// and return to the kernel or the rounds for the LPs behind it.  The verdicts
// match the other path's: non-finite inputs are LP_ERR_INVALID_ARG, some
// b_i < 0 in the max form or some c_j < 0 in the min form
// LP_ERR_INFEASIBLE_START (no Phase I in the server).  An LP the arena cannot
// hold this way goes back to the queue head for the other path.
bool engine_solo(lp_server *sv) {
    Request *r;
    size_t off = 0, bytes = 0;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->fatal != LP_OK || sv->queue.empty()) return false;
        r = &sv->reqs[sv->queue.front()];
        if (!is_solo(sv, *r)) return false;
        bool busy = sv->kernel_running || !sv->active.empty() || sv->busy_lanes > 0;
        for (int s = 0; !busy && s < sv->max_slots; ++s) busy = sv->slot_ticket[s] != 0;
        if (busy) {
            if (!sv->lanes) *(volatile int *)&sv->h_ring->shutdown = 1;
            return false;
        }
        bytes = sv->arena.size();
        if (!sv->arena.alloc(bytes, &off)) return false;
        sv->queue.pop_front();
        r->state = ADMITTED;
        r->t_admit = now_ms();
        r->off = off;
        r->bytes = bytes;
    }
    const int m = r->m, n = r->n;
    const double *A = r->input(), *b = A + (size_t)m * n, *c = b + m;
    const bool resume = r->spilled;
    const bool bneg = !resume && needs_phase1(*r);
    r->x.assign(n, 0.0);
    r->y.assign(m, 0.0);
    double obj = 0.0;
    lp_status st = LP_NOT_SOLVED;
    long long iters = 0;
    lp_err verdict = LP_OK, e = LP_OK;
    lp_handle *h = nullptr;
    bool spilled = false;
    char why[160] = {0};
    if (bneg) {
        verdict = LP_ERR_INFEASIBLE_START;
    } else if (resume) {
        // A spilled LP: its handle's range of the arena back in place (the
        // range starts at the arena's base, where every LP that runs alone
        // starts), then the handle pivots on from where it stopped.
        h = r->solo_h;
        iters = r->iters;  // pivots made before the spill
        // (the whole arena, allocated from empty, starts at offset 0)
        cudaError_t ce = off == 0 ? cudaMemcpyAsync(sv->arena_dev + off, r->host, r->host_used,
                                                    cudaMemcpyHostToDevice, sv->kstream)
                                  : cudaErrorInvalidValue;
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(sv->kstream);
        host_give(sv, r->host, r->host_cap);
        std::lock_guard<std::mutex> lk(sv->mu);
        r->host = nullptr;
        r->spilled = false;
        r->solo_h = nullptr;
        ++sv->restores;
        if (ce != cudaSuccess) {
            e = LP_ERR_CUDA;
            snprintf(why, sizeof why, "restoring a spilled LP: %s", cudaGetErrorString(ce));
        }
    } else {
        if (!sv->solo) {
            lp_options o = sv->opt;
            o.trace_cap = 0;
            o.cuda_stream = nullptr;
            o.time_limit_s = 0.0;
            e = lp_create(&sv->solo, &o);
        }
        h = sv->solo;
        if (e == LP_OK) e = handle_bind_region(h, sv->arena_dev + off, bytes);
        if (e == LP_OK) e = lp_load(h, m, n, A, b, c, (lp_sense)r->sense);
        if (e == LP_OK) r->resident_from = 0;
    }
    // FP64 with spill_pivots: slices of spill_pivots pivots (an FP64 solve
    // cut into calls makes the same pivots, bit for bit); after a slice, when
    // any request is waiting, the LP is spilled and goes to the back of the
    // queue
    const bool sliced = sv->spill_pivots > 0 && !sv->fp32;
    while (h && e == LP_OK && verdict == LP_OK) {
        if (sliced) handle_set_max_iters(h, std::min(sv->spill_pivots, sv->opt.max_iters - iters));
        e = lp_solve(h);
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            ++sv->launches;
        }
        if (e == LP_OK) e = lp_result(h, r->x.data(), r->y.data(), &obj, &st, &iters);
        if (e != LP_OK || !sliced || st != LP_ITER_LIMIT || iters >= sv->opt.max_iters) break;
        bool waiting;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            waiting = !sv->queue.empty();
        }
        if (!waiting) continue;
        const size_t used = handle_region_used(h);
        size_t cap = 0;
        unsigned char *hp = host_take(sv, used, &cap);
        if (!hp) continue;  // no host memory to spill to: pivot on
        cudaError_t ce = cudaMemcpyAsync(hp, sv->arena_dev + off, used, cudaMemcpyDeviceToHost,
                                         sv->kstream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(sv->kstream);
        if (ce != cudaSuccess) {
            host_give(sv, hp, cap);
            e = LP_ERR_CUDA;
            snprintf(why, sizeof why, "spilling an LP: %s", cudaGetErrorString(ce));
            break;
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        r->iters = iters;
        r->host = hp;
        r->host_cap = cap;
        r->host_used = used;
        r->solo_h = h;
        if (h == sv->solo) sv->solo = nullptr;  // the next LP that runs alone takes a new handle
        r->spilled = true;
        ++sv->spills;
        spilled = true;
        break;
    }
    if (e == LP_ERR_INVALID_ARG || e == LP_ERR_INFEASIBLE_START) {
        verdict = e;
        e = LP_OK;
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->arena.release(off, bytes);
    unsigned long long tk = 0;
    for (auto &t : sv->reqs)
        if (&t.second == r) { tk = t.first; break; }
    if (spilled) {
        r->state = QUEUED;
        sv->queue.push_back(tk);
    } else if (e == LP_ERR_OOM && !sv->lanes) {
        r->solo_oom = true;  // the server kernel's slot layout may still hold it
        r->state = QUEUED;
        sv->queue.push_front(tk);
    } else if (e == LP_ERR_OOM) {  // lanes: nothing holds more than the whole arena
        r->err = LP_ERR_OOM;
        r->status = LP_NOT_SOLVED;
        r->state = DONE;
        r->t_done = now_ms();
        ++sv->completed;
    } else if (e != LP_OK) {
        sv->fatal = e;
        snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "server solve of a large LP: %s",
                 why[0] ? why : lp_last_error(h));
    } else {
        r->err = verdict;
        r->status = verdict == LP_OK ? (int)st : LP_NOT_SOLVED;
        r->obj = obj;
        r->iters = iters;
        r->state = DONE;
        r->t_done = now_ms();
        ++sv->completed;
    }
    // inputs loaded (every lp_solve and lp_result waits for the handle's
    // stream) or not needed any more
    if (spilled || r->state == DONE) pin_give(sv, *r);
    // a handle that carried a spilled LP to its end serves the next LP that
    // runs alone, or goes
    if (!spilled && h && h != sv->solo) {
        if (!sv->solo) sv->solo = h;
        else lp_destroy(h);
    }
    *(volatile int *)&sv->h_ring->shutdown = 0;
    sv->cv.notify_all();
    return true;
}

// FP64 lanes (lp_options.lanes > 0): each lane solves one LP at a time, as
// lp_load + lp_solve + lp_result solve it, on its own handle (its own stream,
// SMs / lanes CTAs, its buffers carved from a slice of budget / lanes bytes of
// the arena taken for the LP); the lanes' kernels share the GPU, so the
// chain-bound selection of one LP overlaps the others' updates.  An LP that
// runs alone (solo_elems, or one a slice cannot hold) waits at the head of
// the queue until every lane is idle, the lanes taking no new LP meanwhile,
// then runs on the whole arena and every SM (engine_solo, with its slices and
// spills under spill_pivots).
void lane_main(lp_server *sv) {
    cudaSetDevice(sv->device);
    lp_handle *h = nullptr;
    {
        lp_options o = sv->opt;
        o.trace_cap = 0;
        o.cuda_stream = nullptr;
        o.ctas = sv->lane_ctas;
        o.time_limit_s = 0.0;
        if (lp_create(&h, &o) != LP_OK) {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->fatal = LP_ERR_CUDA;
            snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "lane handle: %s", lp_last_error(nullptr));
            sv->cv.notify_all();
            return;
        }
    }
    while (!sv->stop.load()) {
        Request *r = nullptr;
        unsigned long long tk = 0;
        size_t off = 0;
        bool alone = false;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            if (sv->fatal != LP_OK || sv->queue.empty() || sv->alone_busy) {
                sv->cv.wait_for(lk, std::chrono::microseconds(200));
                continue;
            }
            tk = sv->queue.front();
            Request &q = sv->reqs[tk];
            if (is_solo(sv, q)) {
                if (sv->busy_lanes > 0) {
                    sv->alone_wait = true;
                    sv->cv.wait_for(lk, std::chrono::microseconds(20));
                    continue;
                }
                sv->alone_wait = false;
                sv->alone_busy = true;
                alone = true;
            } else if (sv->alone_wait || !sv->arena.alloc(sv->lane_bytes, &off)) {
                sv->cv.wait_for(lk, std::chrono::microseconds(20));
                continue;
            } else {
                sv->queue.pop_front();
                r = &q;
                r->state = ADMITTED;
                r->t_admit = now_ms();
                ++sv->busy_lanes;
            }
        }
        if (alone) {
            engine_solo(sv);
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->alone_busy = false;
            sv->cv.notify_all();
            continue;
        }
        const int m = r->m, n = r->n;
        const double *A = r->input(), *b = A + (size_t)m * n, *c = b + m;
        r->x.assign(n, 0.0);
        r->y.assign(m, 0.0);
        double obj = 0.0;
        lp_status st = LP_NOT_SOLVED;
        long long iters = 0;
        lp_err e = LP_OK, verdict = LP_OK;
        bool solved = false;
        if (needs_phase1(*r)) {
            verdict = LP_ERR_INFEASIBLE_START;
        } else {
            e = handle_bind_region(h, sv->arena_dev + off, sv->lane_bytes);
            if (e == LP_OK) e = lp_load(h, m, n, A, b, c, (lp_sense)r->sense);
            if (e == LP_OK) {
                e = lp_solve(h);
                solved = true;
            }
            if (e == LP_OK) e = lp_result(h, r->x.data(), r->y.data(), &obj, &st, &iters);
            if (e == LP_ERR_INVALID_ARG || e == LP_ERR_INFEASIBLE_START) {
                verdict = e;
                e = LP_OK;
            }
        }
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->arena.release(off, sv->lane_bytes);
        --sv->busy_lanes;
        if (solved) ++sv->launches;
        if (e == LP_ERR_OOM) {
            r->alone = true;  // a slice cannot hold it: it runs alone
            r->state = QUEUED;
            sv->queue.push_front(tk);
        } else if (e != LP_OK) {
            sv->fatal = e;
            snprintf(sv->fatal_msg, sizeof sv->fatal_msg, "lane solve: %s", lp_last_error(h));
        } else {
            pin_give(sv, *r);
            r->err = verdict;
            r->status = verdict == LP_OK ? (int)st : LP_NOT_SOLVED;
            r->obj = obj;
            r->iters = iters;
            r->state = DONE;
            r->t_done = now_ms();
            ++sv->completed;
        }
        sv->cv.notify_all();
    }
    lp_destroy(h);  // its buffers are the arena's
}

void engine_main(lp_server *sv) {
    cudaSetDevice(sv->device);
    while (!sv->stop.load()) {
        bool progress = engine_complete(sv);
        progress |= engine_admit(sv);
        engine_kernel(sv);
        progress |= engine_solo(sv);
        if (!progress) {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv.wait_for(lk, std::chrono::microseconds(20));
        }
    }
}

}  // namespace

extern "C" {

lp_err lp_server_create(lp_server **out, const lp_options *opt, size_t hbm_budget_bytes,
                        int max_slots) {
    if (!out) return sfail(LP_ERR_INVALID_ARG, "lp_server_create: out is NULL");
    *out = nullptr;
    lp_options o;
    if (opt) o = *opt; else lp_options_default(&o);
    if (o.precision != LP_FP64 && o.precision != LP_FP32_REINV)
        return sfail(LP_ERR_INVALID_ARG, "lp_server_create: unknown precision %d", o.precision);
    if (o.precision == LP_FP32_REINV && o.reinv_k < 1)
        return sfail(LP_ERR_INVALID_ARG, "lp_server_create: reinv_k must be >= 1");
    if (max_slots < 1 || max_slots > kServeMaxSlots || hbm_budget_bytes < (1u << 20))
        return sfail(LP_ERR_INVALID_ARG, "lp_server_create: need 1 <= max_slots <= %d and a "
                     "budget of at least 1 MiB", kServeMaxSlots);
    if (o.max_iters < 0 || o.bland_after < 0 || o.spin_timeout_cycles <= 0 || o.device < 0 ||
        o.spill_pivots < 0 || o.lanes < 0 || o.lanes > 16)
        return sfail(LP_ERR_INVALID_ARG, "lp_server_create: option out of range");
    lp_server *sv = new (std::nothrow) lp_server();
    if (!sv) return sfail(LP_ERR_OOM, "lp_server_create: host allocation failed");
    sv->opt = o;
    sv->device = o.device;
    sv->max_slots = max_slots;
    sv->fp32 = o.precision == LP_FP32_REINV;
    sv->solo_elems = o.solo_elems < 0 ? -1 : o.solo_elems > 0 ? o.solo_elems : 1ll << 24;
    sv->spill_pivots = o.spill_pivots;
    sv->lanes = sv->fp32 ? 0 : o.lanes;
    DeviceRestore restore_;
    cudaError_t e = cudaSetDevice(o.device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sv->sms, cudaDevAttrMultiProcessorCount, o.device);
    const int M = lp_server::kMaxDim + 1, N = 2 * lp_server::kMaxDim + 1;
    sv->smem = (size_t)sv->threads * 2 * sizeof(double) + (((size_t)M * sizeof(double) + 15) & ~(size_t)15) +
               (size_t)std::max(M, N) * sizeof(double);
    if (e == cudaSuccess) {
        sv->ctas = max_coresident_server_ctas(sv->threads, sv->smem, sv->sms);
        sv->workers = sv->ctas - 1;
        if (sv->workers < 1) e = cudaErrorInvalidConfiguration;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->kstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->kdone, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&sv->arena_dev, hbm_budget_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_slots, sizeof(ServeSlot) * max_slots);
    if (e == cudaSuccess) e = cudaMalloc(&sv->d_ctl, sizeof(ServeCtl));
    if (e == cudaSuccess) e = cudaHostAlloc(&sv->h_ring, sizeof(ServeRing), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&sv->d_ring, sv->h_ring, 0);
    if (e == cudaSuccess && sv->fp32) {
        // the batched FP32 launches: a strip of up to threads * 4 floats, the
        // pivot column (FP32) and an FP64 row of the LP's width per CTA
        sv->smem32 = (size_t)sv->threads * 4 * sizeof(float) +
                     (((size_t)M * sizeof(float) + 15) & ~(size_t)15) + (size_t)N * sizeof(double);
        sv->ctas32 = max_coresident_batch_ctas(PREC_FP32, sv->threads, sv->smem32, 1, sv->sms);
        if (sv->ctas32 < 1) e = cudaErrorInvalidConfiguration;
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_desc32, sizeof(LpDesc) * max_slots);
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_desc32, sizeof(LpDesc) * max_slots);
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_items, sizeof(int2) * max_slots * sv->ctas32);
        if (e == cudaSuccess) e = cudaMallocHost(&sv->h_items, sizeof(int2) * max_slots * sv->ctas32);
        if (e == cudaSuccess) e = cudaMalloc(&sv->d_queue, sizeof(unsigned));
        if (e == cudaSuccess) {
            sv->rp = new (std::nothrow) ReinvPool();
            e = sv->rp ? sv->rp->init((size_t)2 * lp_server::kMaxDim) : cudaErrorMemoryAllocation;
        }
        if (e == cudaSuccess) {
            memset(sv->h_desc32, 0, sizeof(LpDesc) * max_slots);
            sv->rule.assign(max_slots, 0);
            sv->failed.assign(max_slots, 0);
            sv->remaining.assign(max_slots, 0);
            sv->guard.assign(max_slots, 0);
            sv->before.assign(max_slots, 0);
        }
    }
    if (e != cudaSuccess) {
        sfail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA, "lp_server_create: %s",
              cudaGetErrorString(e));
        lp_server_destroy(sv);
        return e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA;
    }
    memset(sv->h_ring, 0, sizeof(ServeRing));
    sv->arena.reset(hbm_budget_bytes);
    sv->slot_ticket.assign(max_slots, 0);
    for (int s = max_slots - 1; s >= 0; --s) sv->free_slots.push_back(s);
    if (sv->lanes > 0) {
        sv->lane_ctas = std::max(1, sv->sms / sv->lanes);
        sv->lane_bytes = hbm_budget_bytes / sv->lanes / 256 * 256;
        for (int k = 0; k < sv->lanes; ++k) sv->lane_threads.emplace_back(lane_main, sv);
    } else {
        sv->engine = std::thread(sv->fp32 ? engine32_main : engine_main, sv);
    }
    *out = sv;
    return LP_OK;
}

lp_err lp_server_submit(lp_server *sv, int m, int n, const double *A, const double *b,
                        const double *c, lp_sense sense, unsigned long long *ticket) {
    if (!sv || !A || !b || !c || !ticket)
        return sfail(LP_ERR_INVALID_ARG, "lp_server_submit: NULL argument");
    if (m < 1 || n < 1 || m > lp_server::kMaxDim || n > lp_server::kMaxDim)
        return sfail(LP_ERR_INVALID_ARG, "lp_server_submit: need 1 <= m, n <= %d",
                     lp_server::kMaxDim);
    if (sense != LP_MAX_LE && sense != LP_MIN_GE)
        return sfail(LP_ERR_INVALID_ARG, "lp_server_submit: unknown sense");
    Request r;
    r.m = m;
    r.n = n;
    r.sense = (int)sense;
    int G, W;
    if (sv->fp32) group_shape32(sv, m, n, &G, &W);
    else group_shape(sv, m, n, &G, &W);
    if (slot_layout(m, n, pitch_for(n + m + 1), G, sv->fp32 ? sizeof(float) : sizeof(double)).total >
        sv->arena.size())
        return sfail(LP_ERR_OOM, "lp_server_submit: an LP of %d x %d exceeds the HBM budget", m, n);
    r.nin = (size_t)m * n + m + n;
    double *dst = pin_take(sv, r.nin * sizeof(double), &r.pin_cls);
    r.pin = dst;
    if (!dst) {
        r.in.resize(r.nin);
        dst = r.in.data();
    }
    memcpy(dst, A, sizeof(double) * (size_t)m * n);
    memcpy(dst + (size_t)m * n, b, sizeof(double) * m);
    memcpy(dst + (size_t)m * n + m, c, sizeof(double) * n);
    r.t_submit = now_ms();
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal != LP_OK) {
        pin_give(sv, r);
        return sfail(sv->fatal, "lp_server_submit: %s", sv->fatal_msg);
    }
    const unsigned long long t = sv->next_ticket++;
    sv->reqs.emplace(t, std::move(r));
    sv->queue.push_back(t);
    *ticket = t;
    sv->cv.notify_all();
    return LP_OK;
}

static lp_err take_result(lp_server *sv, std::unordered_map<unsigned long long, Request>::iterator it,
                          double *x, double *y, double *obj, lp_status *status, long long *iters,
                          double *latency_ms) {
    Request &r = it->second;
    if (x) memcpy(x, r.x.data(), sizeof(double) * r.n);
    if (y) memcpy(y, r.y.data(), sizeof(double) * r.m);
    if (obj) *obj = r.obj;
    if (status) *status = (lp_status)r.status;
    if (iters) *iters = r.iters;
    if (latency_ms) *latency_ms = r.t_done - r.t_submit;
    const lp_err e = r.err;
    sv->reqs.erase(it);
    if (e != LP_OK) return sfail(e, "lp_server: request rejected by the input check");
    return LP_OK;
}

lp_err lp_server_poll(lp_server *sv, unsigned long long ticket, int *done, double *x, double *y,
                      double *obj, lp_status *status, long long *iters, double *latency_ms) {
    if (!sv || !done) return sfail(LP_ERR_INVALID_ARG, "lp_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return sfail(LP_ERR_INVALID_ARG, "lp_server_poll: unknown ticket");
    if (it->second.state != DONE) {
        *done = 0;
        if (sv->fatal != LP_OK) return sfail(sv->fatal, "lp_server_poll: %s", sv->fatal_msg);
        return LP_OK;
    }
    *done = 1;
    return take_result(sv, it, x, y, obj, status, iters, latency_ms);
}

lp_err lp_server_wait(lp_server *sv, unsigned long long ticket, double timeout_s, double *x,
                      double *y, double *obj, lp_status *status, long long *iters,
                      double *latency_ms) {
    if (!sv) return sfail(LP_ERR_INVALID_ARG, "lp_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return sfail(LP_ERR_INVALID_ARG, "lp_server_wait: unknown ticket");
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::microseconds((long long)(timeout_s * 1e6));
    while (it->second.state != DONE) {
        if (sv->fatal != LP_OK) return sfail(sv->fatal, "lp_server_wait: %s", sv->fatal_msg);
        if (sv->cv.wait_until(lk, deadline) == std::cv_status::timeout &&
            it->second.state != DONE)
            return sfail(LP_ERR_BUSY, "lp_server_wait: timed out");
        it = sv->reqs.find(ticket);
    }
    return take_result(sv, it, x, y, obj, status, iters, latency_ms);
}

lp_err lp_server_stats(lp_server *sv, long long *completed, long long *launches,
                       size_t *hbm_used, int *queued) {
    if (!sv) return sfail(LP_ERR_INVALID_ARG, "lp_server_stats: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (completed) *completed = sv->completed;
    if (launches) *launches = sv->launches;
    if (hbm_used) *hbm_used = sv->arena.used();
    if (queued) *queued = (int)sv->queue.size();
    return LP_OK;
}

lp_err lp_server_spill_stats(lp_server *sv, long long *spills, long long *restores,
                             size_t *host_bytes) {
    if (!sv) return sfail(LP_ERR_INVALID_ARG, "lp_server_spill_stats: NULL server");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (spills) *spills = sv->spills;
    if (restores) *restores = sv->restores;
    if (host_bytes) *host_bytes = sv->host_total;
    return LP_OK;
}

void lp_server_destroy(lp_server *sv) {
    if (!sv) return;
    sv->stop.store(true);
    sv->cv.notify_all();
    if (sv->engine.joinable()) sv->engine.join();
    for (auto &t : sv->lane_threads)
        if (t.joinable()) t.join();
    DeviceRestore restore_;
    cudaSetDevice(sv->device);
    if (sv->h_ring) *(volatile int *)&sv->h_ring->shutdown = 1;
    if (sv->kstream) cudaStreamSynchronize(sv->kstream);  // the kernel exits once idle
    if (sv->cstream) cudaStreamSynchronize(sv->cstream);
    if (sv->arena_dev) cudaFree(sv->arena_dev);
    if (sv->d_slots) cudaFree(sv->d_slots);
    if (sv->d_ctl) cudaFree(sv->d_ctl);
    if (sv->h_ring) cudaFreeHost(sv->h_ring);
    if (sv->kdone) cudaEventDestroy(sv->kdone);
    if (sv->kstream) cudaStreamDestroy(sv->kstream);
    if (sv->cstream) cudaStreamDestroy(sv->cstream);
    if (sv->d_desc32) cudaFree(sv->d_desc32);
    if (sv->h_desc32) cudaFreeHost(sv->h_desc32);
    if (sv->d_items) cudaFree(sv->d_items);
    if (sv->h_items) cudaFreeHost(sv->h_items);
    if (sv->d_queue) cudaFree(sv->d_queue);
    lp_destroy(sv->solo);  // its buffers are the arena's: nothing of it to free
    for (auto &t : sv->reqs) lp_destroy(t.second.solo_h);  // LPs still spilled
    for (auto &p : sv->host_all) cudaFreeHost(p.first);
    for (void *p : sv->pin_all) cudaFreeHost(p);
    delete sv->rp;
    delete sv;
}

}  // extern "C"
