// Emulated-FP64 matrix products on the tcgen05 tensor cores (an Ozaki-type
// splitting), and the FP32 tableau's body refresh built on them.
//
// GB300 runs FP64 at 2 FMA per clock per SM (1.26 TFLOP/s), but bf16 products
// on the tensor cores at about 2 PFLOP/s.  A product C = A B of FP64 matrices
// is formed from bf16 ones: every row i of A is scaled by sigma_i = 2^e_i
// (|A_ik| < sigma_i) and written as a sum of S = 7 signed 7-bit integer
// digits, A_ik = sigma_i sum_p a_ik^(p) 2^(-7(p+1)) (plus a residual below
// 2^-49 sigma_i); likewise every column j of B with tau_j.  The digits are
// exact in bf16 (|digit| <= 128).  Then
//   C_ij ~= sigma_i tau_j sum_{g=0}^{S-1} 2^(-7(g+2)) G_g,
//   G_g = sum_{p+q=g} sum_k a_ik^(p) b_kj^(q),
// dropping the pairs p + q >= S (below 2^-49 of the scale).  Each G_g is a
// sum of integer products below 2^24 in magnitude for K <= 448 terms, so the
// tensor cores' FP32 accumulation forms it exactly; longer sums are split into
// chunks of 448 whose FP64 results add up.  The epilogue combines the S
// groups in single-single (two-float) arithmetic and scales once in FP64, so
// the FP64 pipe does a few operations per output, not one per group.
//
// Kernel (persistent, 192 threads, one CTA per SM): warp 0 issues the TMA
// loads (cp.async.bulk.tensor, 128-byte swizzle) of the A digit planes (a ring
// of 4 stages of 128 x 64) and of all S B digit planes of a 64-column block
// (two stages); warp 1 issues tcgen05.mma (M 128, N 64, K 16, bf16 in, FP32
// accumulate) for the 28 digit pairs into S accumulators in tensor memory
// (S x 64 of its 512 columns); warps 2-5 read the accumulators (tcgen05.ld) and
// write C.  Every wait is bounded: past the limit a role sets the error flag,
// the others stop at their next wait, the loads in flight are waited for, and
// tensor memory is freed before the CTA exits.
//
// The body refresh (FP32 mode, not in the paper; Sec. 2 Steps 4-5 produce the
// tableau B^-1 [A I b] that it recomputes): with S the structural basic
// variables, R the s rows whose slack is not basic, L the others, and
// Ainv = A_RS^-1 from the Gauss-Jordan step of the reinversion,
//   X = Ainv [A_R | I_R | b_R]            (rows of the structural basics),
//   Y = [A_L | I_L | b_L] - A_LS X        (rows of the slack basics),
// both with the tableau's signs (the dual form enters as -A, -b), rounded into
// the FP32 tableau (basic columns set to exact unit vectors; the rhs column
// and the objective row come from the reinversion's own FP64 values).

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <stdio.h>

#include <algorithm>
#include <mutex>

#include "gbs_device.cuh"
#include "gbs_internal.h"
#include "gbsimplex.h"

namespace gbs {

namespace {

using namespace dev;

constexpr int kOzS = 7;                 // digits per operand
constexpr int kOzT = 7;                 // bits per digit
constexpr int kOzBM = 128, kOzBN = 64, kOzBK = 64;
constexpr int kOzChunkKB = 7;           // K blocks per exact group sum (448 terms)
constexpr int kOzAStages = 4;
constexpr int kOzABytes = kOzBM * kOzBK * 2;            // 16 KB: one A digit plane block
constexpr int kOzBBytes = kOzBN * kOzBK * 2;            // 8 KB: one B digit plane block
constexpr int kOzBStageBytes = kOzS * kOzBBytes;        // 56 KB: all digit planes of a B block
constexpr int kOzTmemCols = 512;                        // S x 64 = 448 used
constexpr int kOzEpiWarps = 16;         // epilogue warps: four per tensor-memory lane quarter
constexpr int kOzThreads = 64 + 32 * kOzEpiWarps;
constexpr size_t kOzSmem = 1024 + 2 * kOzBStageBytes + kOzAStages * kOzABytes + 256;

static_assert(kOzS * kOzBN <= kOzTmemCols, "accumulators must fit tensor memory");
static_assert(kOzT * kOzS == 49, "the digit extraction below assumes 49 bits");

// ---- PTX wrappers ----
__device__ __forceinline__ uint32_t su32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity; false when the limit ran out
// or another CTA or role flagged an error.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int *err, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*(volatile int *)err) return false;
        if (clock64() - t0 > limit) {
            atomicExch(err, 1);
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accum) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
        "%30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand block in the 128-byte
// swizzled layout TMA writes (rows of 128 bytes, 8-row groups 1024 bytes
// apart): start address, stride byte offset 1024, descriptor version 1,
// layout 128-byte swizzle.  The leading byte offset is not used by this
// layout.  Advancing the start address by 32 bytes selects the next 16
// elements of K within the 128-byte row.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) |
           ((uint64_t)(1024 >> 4) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both
// K-major, N = 64, M = 128.
constexpr uint32_t kOzIdesc = (1u << 4) | (1u << 7) | (1u << 10) |
                              ((uint32_t)(kOzBN >> 3) << 17) | ((uint32_t)(kOzBM >> 4) << 24);

// ---- the digits ----
//
// Exponents are biased FP64 exponents shifted by the inner balancing below;
// kNoExp marks a row or column without nonzero entries.  For x = m 2^(ex -
// 1075) (m the 53-bit significand) taken as x 2^sh with |x 2^sh| < 2^(E -
// 1022) (E: the largest shifted exponent of its row or column),
// N = round(x 2^sh 2^(49 - (E - 1022))) is an integer below 2^49 in magnitude,
// and its balanced base-128 digits d_0 .. d_6 (d_0 most significant,
// |d_0| <= 128, the others in [-64, 63]) satisfy
// x 2^sh ~= 2^(E - 1022) sum_p d_p 2^(-7(p+1)).
constexpr int kNoExp = -(1 << 20);

__device__ __forceinline__ int exp_of(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7ff);
}

__device__ __forceinline__ void digits_of(double x, int E, int shift, int (&d)[kOzS]) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7ff);
#pragma unroll
    for (int p = 0; p < kOzS; ++p) d[p] = 0;
    if (ex == 0 || E == kNoExp) return;  // zero (or subnormal, below 2^-1022: dropped)
    const unsigned long long mant = ((unsigned long long)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E - (ex + shift) + 4;  // >= 4
    long long N = 0;
    if (sh < 63) N = (long long)((mant + (1ull << (sh - 1))) >> sh);
    if (b < 0) N = -N;
#pragma unroll
    for (int p = kOzS - 1; p > 0; --p) {
        const long long r = ((N + 64) & 127) - 64;
        d[p] = (int)r;
        N = (N - r) >> 7;
    }
    d[0] = (int)N;
}

// Sources of operand elements.
struct SrcDense {  // p[i * ld + k]
    const double *p;
    long long ld;
    __device__ double at(int i, int k) const { return p[(long long)i * ld + k]; }
};
struct SrcGather {  // sg * A[rows[i]][cols[k]] (A row-major with n columns)
    const double *A;
    int n;
    const int *rows, *cols;
    double sg;
    __device__ double at(int i, int k) const { return sg * A[(long long)rows[i] * n + cols[k]]; }
};
struct SrcRefreshB {  // row r: [sg A_l | e_l | sg b_l], l = R[r]
    const double *A, *b;
    const int *R;
    int n, m;
    double sg;
    __device__ double at(int r, int j) const {
        const int l = R[r];
        if (j < n) return sg * A[(long long)l * n + j];
        if (j < n + m) return (j - n == l) ? 1.0 : 0.0;
        return sg * b[l];
    }
};

// Inner balancing: A B = (A D)(D^-1 B) for D = diag(2^shift_k), exact.  The
// digits keep 49 bits of each row of A and each column of B; when the terms
// of a sum have balanced magnitudes but column k of A and row k of B scale in
// opposite directions (A_RS^-1 times rows of A, with rows of A scaled apart),
// per-row and per-column scales alone would drop whole terms.  shift_k =
// floor((eB_k - eA_k) / 2), with eA_k the largest exponent of column k of A
// and eB_k that of row k of B, brings both to the geometric middle.

// eA_k: largest biased exponent of column k of A (M x K), 0 when the column
// is zero.  A block of 32 x 8 threads takes 32 columns and 64 rows; kA starts
// at 0 and takes each block's maximum by atomicMax.
template <class Src>
__global__ void oz_kexpA_kernel(Src src, int M, int K, int *kA) {
    __shared__ int red[8][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + tx;
    int mx = 0;
    if (k < K) {
        const int i0 = blockIdx.y * 64;
        for (int i = i0 + ty; i < min(M, i0 + 64); i += 8) mx = max(mx, exp_of(src.at(i, k)));
    }
    red[ty][tx] = mx;
    __syncthreads();
    if (ty == 0 && k < K) {
        for (int r = 1; r < 8; ++r) mx = max(mx, red[r][tx]);
        if (mx) atomicMax(kA + k, mx);
    }
}

// eB_k: largest exponent of row k of B (K x N), one warp per k; then shift_k.
template <class Src>
__global__ void oz_kexpB_kernel(Src src, int K, int N, const int *kA, int *shift) {
    const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (k >= K) return;
    int mx = kNoExp;
    for (int j = lane; j < N; j += 32) {
        const int ex = exp_of(src.at(k, j));
        if (ex) mx = max(mx, ex);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) shift[k] = (mx != kNoExp && kA[k] != 0) ? (mx - kA[k]) >> 1 : 0;
}

// Largest shifted exponent of each row i < M of A over k < K (kNoExp: none).
template <class Src>
__global__ void oz_rowexp_kernel(Src src, int M, int K, const int *shift, int *rowexp) {
    const int w = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= M) return;
    int mx = kNoExp;
    for (int k = lane; k < K; k += 32) {
        const int ex = exp_of(src.at(w, k));
        if (ex) mx = max(mx, ex + shift[k]);
    }
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) rowexp[w] = mx;
}

// Largest shifted exponent of each column j < N of B over k < K.
template <class Src>
__global__ void oz_colexp_kernel(Src src, int K, int N, const int *shift, int *colexp) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    int mx = kNoExp;
    for (int k = 0; k < K; ++k) {
        const int ex = exp_of(src.at(k, j));
        if (ex) mx = max(mx, ex - shift[k]);
    }
    colexp[j] = mx;
}

// A digit planes: out[p][i][k] (Mp x Kp per plane), zero in the padding.
template <class Src>
__global__ void oz_split_rows_kernel(Src src, int M, int K, int Mp, int Kp, const int *rowexp,
                                     const int *shift, __nv_bfloat16 *out, int *pmask) {
    const long long total = (long long)Mp * Kp;
    const long long plane = total;
    // (total is a multiple of 32 and Kp of 64: the lanes of a warp stay
    // together and take one row of one 128-row block)
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(e / Kp), k = (int)(e - (long long)i * Kp);
        int d[kOzS];
        if (i < M && k < K) {
            digits_of(src.at(i, k), rowexp[i], shift[k], d);
        } else {
#pragma unroll
            for (int p = 0; p < kOzS; ++p) d[p] = 0;
        }
        unsigned nz = 1u;  // plane 0 always counts (it initialises the accumulators)
#pragma unroll
        for (int p = 0; p < kOzS; ++p) {
            out[p * plane + e] = __float2bfloat16_rn((float)d[p]);
            nz |= d[p] != 0 ? 1u << p : 0u;
        }
        nz = __reduce_or_sync(0xffffffffu, nz);
        if ((threadIdx.x & 31) == 0) atomicOr(pmask + i / kOzBM, (int)nz);
    }
}

// B digit planes, transposed: out[p][j][k] (Np x Kp per plane) for B (K x N),
// through a 32 x 32 tile in shared memory (reads along j, writes along k).
template <class Src>
__global__ void oz_split_cols_kernel(Src src, int K, int N, int Kp, int Np, const int *colexp,
                                     const int *shift, __nv_bfloat16 *out, int *pmask) {
    __shared__ __nv_bfloat16 tile[kOzS][32][33];
    __shared__ int s_nz;
    const int k0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    if (threadIdx.x == 0) s_nz = 1;  // plane 0 always counts
    __syncthreads();
    unsigned nz = 0u;
    for (int r = ty; r < 32; r += 8) {
        const int k = k0 + r, j = j0 + tx;
        int d[kOzS];
        if (k < K && j < N) {
            digits_of(src.at(k, j), colexp[j], -shift[k], d);
        } else {
#pragma unroll
            for (int p = 0; p < kOzS; ++p) d[p] = 0;
        }
#pragma unroll
        for (int p = 0; p < kOzS; ++p) {
            tile[p][r][tx] = __float2bfloat16_rn((float)d[p]);
            nz |= d[p] != 0 ? 1u << p : 0u;
        }
    }
    nz = __reduce_or_sync(0xffffffffu, nz);
    if (tx == 0 && nz) atomicOr(&s_nz, (int)nz);
    __syncthreads();
    // the 32 columns of this block lie in one 64-column block of B
    if (threadIdx.x == 0) atomicOr(pmask + j0 / kOzBN, s_nz);
    const size_t plane = (size_t)Np * Kp;
    for (int r = ty; r < 32; r += 8) {
        const int j = j0 + r, k = k0 + tx;
        if (j < Np && k < Kp) {
#pragma unroll
            for (int p = 0; p < kOzS; ++p) out[p * plane + (size_t)j * Kp + k] = tile[p][tx][r];
        }
    }
}

__device__ __forceinline__ void named_bar(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// A named barrier that also ANDs a flag over its threads, so that they all
// take the same branch after it.
__device__ __forceinline__ bool named_bar_and(int id, int nthreads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\n"
        "bar.red.and.pred q, %2, %3, p;\nselp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(id), "r"(nthreads)
        : "memory");
    return r != 0;
}

// ---- the product kernel ----
struct OzParams {
    int M, N, K, Mp, Np, Kp;
    const int *rowexp, *colexp;
    // digit planes with a nonzero digit, per 128-row block of A and per
    // 64-column block of B (bit p: plane p; plane 0 always set)
    const int *amask, *bmask;
    int mode;  // 0: C = A B (FP64, rows < M, cols < N); 1: refresh rows into the FP32 tableau
    double *C;
    long long ldc;
    // mode 1: output row r is tableau row rowmap[r], constraint rowk[r]; the
    // value written is sg [A_k | e_k](j) - (A B)_rj for j < N, with the
    // basic columns set to unit vectors (basic_row[j]: the row where column j
    // is basic, or -1)
    float *T32;
    long long P;
    const int *rowmap, *rowk, *basic_row;
    const double *Aorig;
    int n, m;
    double sg;
    int *err;
    unsigned long long *mmas;  // += the tcgen05.mma instructions issued (128 x 64 x 16 each)
    long long spin_limit;
};

__device__ __forceinline__ float pow2f(int e) {  // 2^e, e in [-126, 127]
    return __int_as_float((e + 127) << 23);
}
// f 2^e as a double, assembled from the bits (exact; no FP64 instruction);
// false when f is subnormal or the result leaves the normal FP64 range.
__device__ __forceinline__ bool f2d_scaled(float f, int e, double &out) {
    const unsigned u = __float_as_uint(f);
    const int fe = (int)((u >> 23) & 0xffu);
    if (fe == 0) {
        out = 0.0;
        return (u & 0x7fffffu) == 0u;
    }
    const int de = fe - 127 + 1023 + e;
    if (de < 1 || de > 2046) return false;
    out = __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) |
                                           ((unsigned long long)de << 52) |
                                           ((unsigned long long)(u & 0x7fffffu) << 29)));
    return true;
}

// (hi + lo) 2^e outside the normal range (rare; kept out of line)
__device__ __noinline__ double scaled_sum_slow(float hi, float lo, int e) {
    return ldexp((double)hi + (double)lo, e);
}
// sigma_r tau_j 2^-14 (hi + lo): two exact conversions and one FP64 add.
__device__ __forceinline__ double scaled_sum(float hi, float lo, int e) {
    double dh, dl;
    if (f2d_scaled(hi, e, dh) && f2d_scaled(lo, e, dl)) return dh + dl;
    return scaled_sum_slow(hi, lo, e);
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__global__ void __launch_bounds__(kOzThreads, 1)
    oz_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const OzParams p) {
    extern __shared__ unsigned char oz_smem[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_colexp[kOzBN], s_brow[kOzBN];
    const uint32_t raw = su32(oz_smem);
    const uint32_t base = (raw + 1023u) & ~1023u;
    const uint32_t sB = base;                                  // [2][S][64][128 B]
    const uint32_t sA = base + 2 * kOzBStageBytes;             // [4][128][128 B]
    const uint32_t sBar = sA + kOzAStages * kOzABytes;         // barriers, 8 bytes each
    auto full_a = [&](int s) { return sBar + 8u * s; };
    auto empty_a = [&](int s) { return sBar + 8u * (kOzAStages + s); };
    auto full_b = [&](int s) { return sBar + 8u * (2 * kOzAStages + s); };
    auto empty_b = [&](int s) { return sBar + 8u * (2 * kOzAStages + 2 + s); };
    const uint32_t tmem_full = sBar + 8u * (2 * kOzAStages + 4);
    const uint32_t tmem_empty = sBar + 8u * (2 * kOzAStages + 5);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzAStages; ++s) {
            mbar_init(full_a(s), 1);
            mbar_init(empty_a(s), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(full_b(s), 1);
            mbar_init(empty_b(s), 1);
        }
        mbar_init(tmem_full, 1);
        mbar_init(tmem_empty, kOzEpiWarps);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&s_tmem)),
                     "r"(kOzTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    const int nmb = p.Mp / kOzBM, nnb = p.Np / kOzBN, tiles = nmb * nnb;
    const int nkb = p.Kp / kOzBK;
    const int nch = (nkb + kOzChunkKB - 1) / kOzChunkKB;
    const long long lim = p.spin_limit;

    if (warp == 0) {
        // ---- TMA producer ----
        if (lane == 0) {
            int as = 0, bs = 0;
            uint32_t aph = 0, bph = 0;
            // loads issued and not yet seen complete, per stage, for the drain
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int m0 = (t % nmb) * kOzBM, n0 = (t / nmb) * kOzBN;
                // planes that are zero for the whole row (column) block are
                // neither loaded nor multiplied
                const int ma = p.amask[m0 / kOzBM], mb = p.bmask[n0 / kOzBN];
                for (int kb = 0; kb < nkb && ok; ++kb) {
                    if (!(ok = mbar_wait(empty_b(bs), bph ^ 1u, p.err, lim))) break;
                    mbar_expect_tx(full_b(bs), (uint32_t)(__popc(mb) * kOzBBytes));
                    for (int q = 0; q < kOzS; ++q)
                        if ((mb >> q) & 1)
                            tma_load_2d(sB + bs * kOzBStageBytes + q * kOzBBytes, &tmB, kb * kOzBK,
                                        q * p.Np + n0, full_b(bs));
                    if (++bs == 2) {
                        bs = 0;
                        bph ^= 1u;
                    }
                    for (int pp = 0; pp < kOzS; ++pp) {
                        if (!((ma >> pp) & 1)) continue;
                        if (!(ok = mbar_wait(empty_a(as), aph ^ 1u, p.err, lim))) break;
                        mbar_expect_tx(full_a(as), kOzABytes);
                        tma_load_2d(sA + as * kOzABytes, &tmA, kb * kOzBK, pp * p.Mp + m0, full_a(as));
                        if (++as == kOzAStages) {
                            as = 0;
                            aph ^= 1u;
                        }
                    }
                }
            }
            if (!ok) {
                // Drain: every load issued completes on its stage's full
                // barrier; wait (bounded) for the phase each stage is in, so
                // that no copy still writes shared memory when the CTA ends.
                for (int s = 0; s < kOzAStages; ++s) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(full_a(s), ((s < as) ? aph : aph ^ 1u)) && clock64() - t0 < lim) {}
                }
                for (int s = 0; s < 2; ++s) {
                    const long long t0 = clock64();
                    while (!mbar_try_wait(full_b(s), ((s < bs) ? bph : bph ^ 1u)) && clock64() - t0 < lim) {}
                }
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            int as = 0, bs = 0;
            uint32_t aph = 0, bph = 0, use = 0;
            unsigned long long nmma = 0;  // MMA instructions issued
            bool ok = true;
            for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
                const int ma = p.amask[(t % nmb)], mb = p.bmask[(t / nmb)];
                for (int c = 0; c < nch && ok; ++c) {
                    // the epilogue has drained the accumulators of the last use
                    if (!(ok = mbar_wait(tmem_empty, (use & 1u) ^ 1u, p.err, lim))) break;
                    tc_fence_after();
                    const int kb0 = c * kOzChunkKB, kb1 = min(nkb, kb0 + kOzChunkKB);
                    uint32_t inited = 0u;  // accumulator groups written in this chunk
                    for (int kb = kb0; kb < kb1 && ok; ++kb) {
                        // (TMA-written shared memory is read by the MMAs, both
                        // async-proxy operations: the barrier wait orders them)
                        if (!(ok = mbar_wait(full_b(bs), bph, p.err, lim))) break;
                        // descriptors: B digit plane q of this stage is 8 KB
                        // (512 descriptor units) after plane 0; each K step of 16
                        // elements advances a descriptor by 32 bytes (2 units)
                        const uint64_t bd0 = sw128_desc(sB + bs * kOzBStageBytes);
                        for (int pp = 0; pp < kOzS; ++pp) {
                            if (!((ma >> pp) & 1)) continue;
                            if (!(ok = mbar_wait(full_a(as), aph, p.err, lim))) break;
                            const uint64_t ad = sw128_desc(sA + as * kOzABytes);
#pragma unroll
                            for (int q = 0; q < kOzS; ++q) {
                                if (q < kOzS - pp && ((mb >> q) & 1)) {
                                    // the first product into a group of this chunk
                                    // overwrites it
                                    const uint32_t acc0 = (inited >> (pp + q)) & 1u;
                                    inited |= 1u << (pp + q);
                                    const uint32_t d = tmem + (uint32_t)((pp + q) * kOzBN);
                                    const uint64_t bd = bd0 + (uint64_t)(q * (kOzBBytes >> 4));
                                    tc_mma(d, ad, bd, kOzIdesc, acc0);
                                    tc_mma(d, ad + 2, bd + 2, kOzIdesc, 1u);
                                    tc_mma(d, ad + 4, bd + 4, kOzIdesc, 1u);
                                    tc_mma(d, ad + 6, bd + 6, kOzIdesc, 1u);
                                    nmma += 4;
                                }
                            }
                            tc_commit(empty_a(as));  // the stage frees when these MMAs complete
                            if (++as == kOzAStages) {
                                as = 0;
                                aph ^= 1u;
                            }
                        }
                        if (!ok) break;
                        tc_commit(empty_b(bs));
                        if (++bs == 2) {
                            bs = 0;
                            bph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_commit(tmem_full);
                    ++use;
                }
            }
            if (p.mmas) atomicAdd(p.mmas, nmma);
            // every MMA issued is complete before tensor memory is freed
            // (a commit arrives after all of them)
            if (!ok) {
                tc_commit(tmem_full);
                const long long t0 = clock64();
                while (!mbar_try_wait(tmem_full, use & 1u) && clock64() - t0 < lim) {}
            }
        }
    } else {
        // ---- epilogue: warps 2..17, TMEM lanes 32 (warp % 4) .. + 31; warps
        // 2..5 take the tile's columns 0..15, warps 6..9 columns 16..31, and so on ----
        const int lg = warp & 3, et = threadIdx.x - 64, hsel = (warp - 2) >> 2;
        uint32_t use = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
            const int m0 = (t % nmb) * kOzBM, n0 = (t / nmb) * kOzBN;
            const int r = m0 + lg * 32 + lane;  // this thread's output row
            for (int c = 0; c < nch && ok; ++c) {
                // all the epilogue warps leave together or go on together
                // (this barrier also follows the previous tile's reads of
                // the shared column data)
                ok = named_bar_and(1, 32 * kOzEpiWarps, mbar_wait(tmem_full, use & 1u, p.err, lim));
                if (!ok) break;
                tc_fence_after();
                const int Er = r < p.M ? p.rowexp[r] : kNoExp;
                // the tile's column exponents (and basic rows) in shared
                // memory, read by every lane at once (a broadcast)
                if (et < kOzBN) {
                    const int col = n0 + et;
                    s_colexp[et] = col < p.N ? p.colexp[col] : kNoExp;
                    if (p.mode == 1) s_brow[et] = col < p.N - 1 ? p.basic_row[col] : -1;
                }
                named_bar(1, 32 * kOzEpiWarps);
                const uint32_t tbase = tmem + ((uint32_t)(lg * 32) << 16);
                // the accumulator groups the MMA issuer wrote for this tile
                uint32_t gm = 0u;
                {
                    const int ma = p.amask[m0 / kOzBM], mb = p.bmask[n0 / kOzBN];
                    for (int pa = 0; pa < kOzS; ++pa)
                        if ((ma >> pa) & 1)
                            for (int qb = 0; qb < kOzS - pa; ++qb)
                                if ((mb >> qb) & 1) gm |= 1u << (pa + qb);
                }
                {
                    // the warp's 16 columns in two blocks of 8 (few enough
                    // registers for four epilogue warps per lane quarter)
                    int ti = 0, kr = 0;  // mode 1: this row's place in the tableau, its constraint
                    if (p.mode == 1 && r < p.M) {
                        ti = p.rowmap[r];
                        kr = p.rowk[r];
                    }
                    const double *arow = p.Aorig + (long long)kr * p.n;
#pragma unroll 1
                    for (int sb = 0; sb < 2; ++sb) {
                        const int cb = hsel * 16 + sb * 8;  // the block's first column in the tile
                        const int j0 = n0 + cb;
                        // mode 1: the row's original entries at the block's
                        // columns, read before the accumulators so that their
                        // latency overlaps the reads of tensor memory
                        double av[8];
                        if (p.mode == 1 && r < p.M) {
#pragma unroll
                            for (int j = 0; j < 8; ++j) av[j] = j0 + j < p.n ? __ldg(arow + j0 + j) : 0.0;
                        }
                        float hi[8], lo[8];
#pragma unroll
                        for (int g = 0; g < kOzS; ++g) {
                            uint32_t v[8];
                            tmem_ld8(tbase + (uint32_t)(g * kOzBN + cb), v);
                            tmem_ld_wait();
                            const float sc = pow2f(-kOzT * g);
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                // (a group no digit pair wrote holds stale columns: zero)
                                const float x = ((gm >> g) & 1u)
                                                    ? __fmul_rn(__uint_as_float(v[j]), sc)  // exact
                                                    : 0.0f;
                                if (g == 0) {
                                    hi[j] = x;
                                    lo[j] = 0.0f;
                                } else {
                                    float s, e;
                                    two_sum(hi[j], x, s, e);
                                    hi[j] = s;
                                    lo[j] = __fadd_rn(lo[j], e);
                                }
                            }
                        }
                        if (sb == 1) {
                            // this warp's accumulators are in registers: once every
                            // epilogue warp's are, the MMAs of the next tile may
                            // start while the results are written
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) mbar_arrive(tmem_empty);
                        }
                        // Each thread writes its own row's results (the row its
                        // tensor-memory lane holds): one contiguous row segment per
                        // thread, read (C, or the original row of A) and written with
                        // independent accesses, no shared-memory transposition.
                        if (p.mode == 0) {
                            if (r < p.M) {
                                double *crow = p.C + (long long)r * p.ldc + j0;
#pragma unroll
                                for (int j = 0; j < 8; ++j) {
                                    const int Fc = s_colexp[cb + j];
                                    double v = 0.0;
                                    // scale 2^(Er - 1022 + Fc - 1022 - 14)
                                    if (Er != kNoExp && Fc != kNoExp) v = scaled_sum(hi[j], lo[j], Er + Fc - 2058);
                                    if (j0 + j < p.N) crow[j] = c == 0 ? v : crow[j] + v;
                                }
                            }
                        } else if (r < p.M) {
                            const long long sgbit = p.sg < 0.0 ? (long long)kSign : 0ll;
                            float *trow = p.T32 + (long long)ti * p.P;
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                const int col = j0 + j;
                                // the rhs column comes from the reinversion
                                if (col < p.N - 1) {
                                    const int br = s_brow[cb + j];
                                    float out;
                                    if (br >= 0) {
                                        out = br == ti ? 1.0f : 0.0f;
                                    } else {
                                        const int Fc = s_colexp[cb + j];
                                        double v = 0.0;
                                        if (Er != kNoExp && Fc != kNoExp) v = scaled_sum(hi[j], lo[j], Er + Fc - 2058);
                                        // sg A_kj by its sign bit (no FP64 multiply)
                                        const double d = col < p.n ? __longlong_as_double(__double_as_longlong(av[j]) ^ sgbit)
                                                                   : (col - p.n == kr ? 1.0 : 0.0);
                                        out = __double2float_rn(d - v);
                                    }
                                    trow[col] = out;
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
                ++use;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kOzTmemCols)
                     : "memory");
    }
}

// ---- host side ----
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// A 2D map over `rows` rows of `Kp` bf16 (row pitch Kp * 2 bytes), boxes of
// 64 x box_rows, 128-byte swizzle.
cudaError_t make_map(CUtensorMap *map, void *ptr, long long rows, int Kp, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kOzBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, ptr, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Grow a workspace buffer to hold n elements of T (contents not kept).
template <class T>
cudaError_t grow_buf(T **p, size_t *cap, size_t n) {
    if (*cap >= n && *p) return cudaSuccess;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e == cudaSuccess) *cap = n;
    return e;
}
cudaError_t grow_planes(void **p, size_t *cap, size_t n) {
    __nv_bfloat16 *q = static_cast<__nv_bfloat16 *>(*p);
    const cudaError_t e = grow_buf(&q, cap, n);
    *p = q;
    return e;
}

int round_up(int x, int a) { return (x + a - 1) / a * a; }

// Grow the digit planes and exponent arrays for an M x K by K x N product.
cudaError_t oz_reserve(OzWork &w, int M, int N, int K) {
    const int Mp = round_up(std::max(M, 1), kOzBM), Np = round_up(std::max(N, 1), kOzBN),
              Kp = round_up(std::max(K, 1), kOzBK);
    cudaError_t e;
    if ((e = grow_planes(&w.asl, &w.cap_asl, (size_t)kOzS * Mp * Kp)) != cudaSuccess) return e;
    if ((e = grow_planes(&w.bsl, &w.cap_bsl, (size_t)kOzS * Np * Kp)) != cudaSuccess) return e;
    if ((e = grow_buf(&w.rowexp, &w.cap_rowexp, (size_t)std::max(M, 1))) != cudaSuccess) return e;
    if ((e = grow_buf(&w.colexp, &w.cap_colexp, (size_t)std::max(N, 1))) != cudaSuccess) return e;
    if ((e = grow_buf(&w.kx, &w.cap_kx, (size_t)2 * std::max(K, 1))) != cudaSuccess) return e;
    if ((e = grow_buf(&w.pmask, &w.cap_pmask, (size_t)(Mp / kOzBM + Np / kOzBN))) != cudaSuccess)
        return e;
    if (!w.err && (e = cudaMalloc((void **)&w.err, sizeof(int))) != cudaSuccess) return e;
    if (!w.mmas && (e = cudaMalloc((void **)&w.mmas, sizeof(unsigned long long))) != cudaSuccess)
        return e;
    return cudaSuccess;
}

// Digits of A (M x K from srcA) and B (K x N from srcB), then the product.
// The workspace must already hold this size (oz_reserve): growing it here
// could free a buffer that queued work still reads.
template <class SA, class SB>
cudaError_t oz_product(SA srcA, SB srcB, int M, int N, int K, OzParams p, OzWork &w, int sms,
                       cudaStream_t s) {
    const int Mp = round_up(std::max(M, 1), kOzBM), Np = round_up(std::max(N, 1), kOzBN),
              Kp = round_up(std::max(K, 1), kOzBK);
    cudaError_t e;
    if (w.cap_asl < (size_t)kOzS * Mp * Kp || w.cap_bsl < (size_t)kOzS * Np * Kp ||
        w.cap_rowexp < (size_t)M || w.cap_colexp < (size_t)N || w.cap_kx < (size_t)2 * K ||
        w.cap_pmask < (size_t)(Mp / kOzBM + Np / kOzBN) || !w.err || !w.mmas)
        return cudaErrorInvalidValue;
    int *kA = w.kx, *shift = w.kx + K;
    int *amask = w.pmask, *bmask = w.pmask + Mp / kOzBM;
    if ((e = cudaMemsetAsync(w.pmask, 0, sizeof(int) * (size_t)(Mp / kOzBM + Np / kOzBN), s)) !=
        cudaSuccess)
        return e;
    if (K > 0) {
        if ((e = cudaMemsetAsync(kA, 0, sizeof(int) * (size_t)K, s)) != cudaSuccess) return e;
        oz_kexpA_kernel<SA><<<dim3((K + 31) / 32, (M + 63) / 64), 256, 0, s>>>(srcA, M, K, kA);
        oz_kexpB_kernel<SB><<<(K + 7) / 8, 256, 0, s>>>(srcB, K, N, kA, shift);
    }
    oz_rowexp_kernel<SA><<<(M + 7) / 8, 256, 0, s>>>(srcA, M, K, shift, w.rowexp);
    oz_colexp_kernel<SB><<<(N + 255) / 256, 256, 0, s>>>(srcB, K, N, shift, w.colexp);
    {
        const long long total = (long long)Mp * Kp;
        const int blocks = (int)std::min<long long>((total + 255) / 256, 8LL * sms * 8);
        oz_split_rows_kernel<SA><<<blocks, 256, 0, s>>>(srcA, M, K, Mp, Kp, w.rowexp, shift,
                                                         static_cast<__nv_bfloat16 *>(w.asl), amask);
    }
    oz_split_cols_kernel<SB><<<dim3(Np / 32, Kp / 32), 256, 0, s>>>(
        srcB, K, N, Kp, Np, w.colexp, shift, static_cast<__nv_bfloat16 *>(w.bsl), bmask);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    CUtensorMap ma, mb;
    if ((e = make_map(&ma, w.asl, (long long)kOzS * Mp, Kp, kOzBM)) != cudaSuccess) return e;
    if ((e = make_map(&mb, w.bsl, (long long)kOzS * Np, Kp, kOzBN)) != cudaSuccess) return e;
    p.M = M;
    p.N = N;
    p.K = K;
    p.Mp = Mp;
    p.Np = Np;
    p.Kp = Kp;
    p.rowexp = w.rowexp;
    p.colexp = w.colexp;
    p.amask = amask;
    p.bmask = bmask;
    if (!p.err) p.err = w.err;
    p.mmas = w.mmas;
    if ((e = cudaMemsetAsync(p.err, 0, sizeof(int), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.mmas, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    if (p.mode == 1 && Kp > kOzChunkKB * kOzBK) return cudaErrorInvalidValue;  // one chunk only
    if ((e = cudaFuncSetAttribute(oz_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kOzSmem)) != cudaSuccess)
        return e;
    const int tiles = (Mp / kOzBM) * (Np / kOzBN);
    oz_gemm_kernel<<<std::min(tiles, sms), kOzThreads, kOzSmem, s>>>(ma, mb, p);
    return cudaGetLastError();
}

}  // namespace

void oz_work_free(OzWork &w) {
    void *ps[] = {w.asl, w.bsl, w.rowexp, w.colexp, w.kx, w.pmask, w.X, w.Ainv, w.Z, w.basic_row, w.L, w.Lrow, w.err,
                  w.mmas};
    for (void *q : ps)
        if (q) cudaFree(q);
    w = OzWork{};
}

cudaError_t oz_dgemm(const double *A, long long lda, const double *B, long long ldb, double *C,
                     long long ldc, int M, int N, int K, OzWork &w, int *d_err, int sms,
                     long long spin_limit, cudaStream_t s) {
    cudaError_t e = oz_reserve(w, M, N, K);
    if (e != cudaSuccess) return e;
    OzParams p{};
    p.mode = 0;
    p.C = C;
    p.ldc = ldc;
    p.err = d_err;
    p.spin_limit = spin_limit;
    return oz_product(SrcDense{A, lda}, SrcDense{B, ldb}, M, N, K, p, w, sms, s);
}

namespace {

// Ainv[k][r] = row k of A_RS^-1, which the Gauss-Jordan step leaves in row
// pivrow[k] of the right block of W = [A_RS | b_R | I].
__global__ void oz_ainv_kernel(const double *__restrict__ W, long long Wp, int ns,
                               const int *__restrict__ pivrow, double *__restrict__ Ainv) {
    const long long total = (long long)ns * ns;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / ns), r = (int)(e - (long long)k * ns);
        Ainv[e] = W[(long long)pivrow[k] * Wp + ns + 1 + r];
    }
}

// basic_row[v] = the row where variable v is basic (the array starts at -1).
__global__ void oz_basic_kernel(const int *__restrict__ basis, int m, int *__restrict__ basic_row) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) basic_row[basis[i]] = i;
}

// L = the constraints whose slack is basic, ascending; Lrow[r] = the row
// where the slack of L[r] is basic (one CTA of 1024 threads).
__global__ void __launch_bounds__(1024) oz_llist_kernel(const int *__restrict__ basic_row, int m,
                                                        int n, int *__restrict__ L,
                                                        int *__restrict__ Lrow) {
    __shared__ int scan[1024];
    const int tid = threadIdx.x, B = blockDim.x;
    const int chunk = (m + B - 1) / B;
    const int l0 = min(m, tid * chunk), l1 = min(m, l0 + chunk);
    int cnt = 0;
    for (int l = l0; l < l1; ++l) cnt += basic_row[n + l] >= 0;
    scan[tid] = cnt;
    __syncthreads();
    for (int o = 1; o < B; o <<= 1) {
        const int a = tid >= o ? scan[tid - o] : 0;
        __syncthreads();
        scan[tid] += a;
        __syncthreads();
    }
    int k = scan[tid] - cnt;
    for (int l = l0; l < l1; ++l) {
        const int r = basic_row[n + l];
        if (r >= 0) {
            L[k] = l;
            Lrow[k] = r;
            ++k;
        }
    }
}

// The rows of the structural basics: tableau row basic_row[S[k]] = X[k] in
// FP32, basic columns as unit vectors, every column but the rhs.
__global__ void oz_xrows_kernel(const double *__restrict__ X, int N, int ns, const int *__restrict__ S,
                                const int *__restrict__ basic_row, float *__restrict__ T32, long long P) {
    const long long total = (long long)ns * (N - 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(e / (N - 1)), j = (int)(e - (long long)k * (N - 1));
        const int ti = basic_row[S[k]], br = basic_row[j];
        T32[(long long)ti * P + j] = br >= 0 ? (br == ti ? 1.0f : 0.0f) : (float)X[(long long)k * N + j];
    }
}

// The rows of the slack basics from Z = A_LS X (when the product took more
// than one K chunk): sg [A_l | e_l](j) - Z[r][j].
__global__ void oz_yrows_kernel(const double *__restrict__ Z, int N, int mL, const int *__restrict__ L,
                                const int *__restrict__ Lrow, const double *__restrict__ A, int n,
                                double sg, const int *__restrict__ basic_row, float *__restrict__ T32,
                                long long P) {
    const long long total = (long long)mL * (N - 1);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e / (N - 1)), j = (int)(e - (long long)r * (N - 1));
        const int ti = Lrow[r], l = L[r], br = basic_row[j];
        float v;
        if (br >= 0) {
            v = br == ti ? 1.0f : 0.0f;
        } else {
            const double d = j < n ? sg * A[(long long)l * n + j] : (j - n == l ? 1.0 : 0.0);
            v = (float)(d - Z[(long long)r * N + j]);
        }
        T32[(long long)ti * P + j] = v;
    }
}

int grid_for(long long total) {
    return (int)std::max<long long>(1, std::min<long long>((total + 255) / 256, 4096));
}

}  // namespace

cudaError_t oz_refresh_body(const double *A, const double *b, int sense, int m, int n,
                            const int *basis, const ReinvBufs &rb, int ns, float *T32,
                            long long P, OzWork &w, int sms, long long spin_limit,
                            cudaStream_t s) {
    const double sg = sense == 0 ? 1.0 : -1.0;
    const int N = n + m + 1, mL = m - ns;
    const bool one_chunk = round_up(std::max(ns, 1), kOzBK) <= kOzChunkKB * kOzBK;
    cudaError_t e;
    // every buffer at its final size before any work is queued
    if ((e = grow_buf(&w.basic_row, &w.cap_basic, (size_t)(n + m))) != cudaSuccess) return e;
    if ((e = grow_buf(&w.L, &w.cap_L, (size_t)m)) != cudaSuccess) return e;
    if ((e = grow_buf(&w.Lrow, &w.cap_Lrow, (size_t)m)) != cudaSuccess) return e;
    if ((e = grow_buf(&w.X, &w.cap_X, (size_t)ns * N)) != cudaSuccess) return e;
    if ((e = grow_buf(&w.Ainv, &w.cap_Ainv, (size_t)ns * ns)) != cudaSuccess) return e;
    if (!one_chunk && (e = grow_buf(&w.Z, &w.cap_Z, (size_t)mL * N)) != cudaSuccess) return e;
    if ((e = oz_reserve(w, ns, N, ns)) != cudaSuccess) return e;
    if ((e = oz_reserve(w, mL, N, ns)) != cudaSuccess) return e;

    if ((e = cudaMemsetAsync(w.basic_row, 0xff, sizeof(int) * (size_t)(n + m), s)) != cudaSuccess)
        return e;
    oz_basic_kernel<<<(m + 255) / 256, 256, 0, s>>>(basis, m, w.basic_row);
    oz_llist_kernel<<<1, 1024, 0, s>>>(w.basic_row, m, n, w.L, w.Lrow);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (ns > 0) {
        oz_ainv_kernel<<<grid_for((long long)ns * ns), 256, 0, s>>>(rb.W, rb.Wp, ns, rb.pivrow, w.Ainv);
        OzParams p{};
        p.mode = 0;
        p.C = w.X;
        p.ldc = N;
        p.spin_limit = spin_limit;
        e = oz_product(SrcDense{w.Ainv, ns}, SrcRefreshB{A, b, rb.R, n, m, sg}, ns, N, ns, p, w,
                       sms, s);
        if (e != cudaSuccess) return e;
        oz_xrows_kernel<<<grid_for((long long)ns * (N - 1)), 256, 0, s>>>(w.X, N, ns, rb.S,
                                                                           w.basic_row, T32, P);
    }
    if (mL > 0) {
        OzParams p{};
        p.spin_limit = spin_limit;
        const SrcGather a2{A, n, w.L, rb.S, sg};
        if (one_chunk) {
            p.mode = 1;
            p.T32 = T32;
            p.P = P;
            p.rowmap = w.Lrow;
            p.rowk = w.L;
            p.basic_row = w.basic_row;
            p.Aorig = A;
            p.n = n;
            p.m = m;
            p.sg = sg;
            e = oz_product(a2, SrcDense{w.X, N}, mL, N, ns, p, w, sms, s);
        } else {
            p.mode = 0;
            p.C = w.Z;
            p.ldc = N;
            e = oz_product(a2, SrcDense{w.X, N}, mL, N, ns, p, w, sms, s);
            if (e == cudaSuccess)
                oz_yrows_kernel<<<grid_for((long long)mL * (N - 1)), 256, 0, s>>>(
                    w.Z, N, mL, w.L, w.Lrow, A, n, sg, w.basic_row, T32, P);
        }
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

}  // namespace gbs

namespace {
constexpr int kOzMaxDevices = 64;
std::mutex g_oz_mutex;
gbs::OzWork g_oz_work[kOzMaxDevices];
long long g_oz_last_mmas = 0;  // MMAs of the last lp_dgemm_emulated (under g_oz_mutex)
}  // namespace

extern "C" lp_err lp_dgemm_emulated(int M, int N, int K, const double *A, long long lda,
                                    const double *B, long long ldb, double *C, long long ldc,
                                    const lp_options *opt) {
    using namespace gbs;
    char msg[256];
    if (M < 1 || N < 1 || K < 1 || !A || !B || !C || lda < K || ldb < N || ldc < N) {
        set_last_error_global("lp_dgemm_emulated: need M, N, K >= 1, non-NULL A, B, C and "
                              "lda >= K, ldb >= N, ldc >= N");
        return LP_ERR_INVALID_ARG;
    }
    lp_options o;
    if (opt) o = *opt; else lp_options_default(&o);
    const void *ptrs[] = {A, B, C};
    for (const void *q : ptrs) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess ||
            (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
            cudaGetLastError();
            set_last_error_global("lp_dgemm_emulated: A, B and C must be device memory");
            return LP_ERR_INVALID_ARG;
        }
    }
    DeviceRestore restore_;
    cudaError_t e = cudaSetDevice(o.device);
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, o.device);
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    if (o.device < 0 || o.device >= kOzMaxDevices) {
        set_last_error_global("lp_dgemm_emulated: device out of range");
        return LP_ERR_INVALID_ARG;
    }
    // one workspace per device, kept between calls (it only grows), so that
    // repeated products allocate nothing; calls are serialised
    std::lock_guard<std::mutex> lock(g_oz_mutex);
    OzWork &w = g_oz_work[o.device];
    int herr = 0;
    unsigned long long nmma = 0;
    if (e == cudaSuccess)
        e = oz_dgemm(A, lda, B, ldb, C, ldc, M, N, K, w, nullptr, sms, o.spin_timeout_cycles, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, w.err, sizeof herr, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nmma, w.mmas, sizeof nmma, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    g_oz_last_mmas = e == cudaSuccess ? (long long)nmma : 0;
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "lp_dgemm_emulated: %s", cudaGetErrorString(e));
        set_last_error_global(msg);
        return LP_ERR_CUDA;
    }
    if (herr) {
        set_last_error_global("lp_dgemm_emulated: a device wait ran out (spin_timeout_cycles)");
        return LP_ERR_CUDA;
    }
    return LP_OK;
}

extern "C" lp_err lp_dgemm_stats(long long *tensor_mmas) {
    if (!tensor_mmas) {
        gbs::set_last_error_global("lp_dgemm_stats: NULL output");
        return LP_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_oz_mutex);
    *tensor_mmas = g_oz_last_mmas;
    return LP_OK;
}
