// Shared device/host helpers of libosvmbe (GB300, sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

namespace osv {

constexpr int kWarp = 32;

// Process-wide count of kernel launches issued by this library (osv_kernel_launches).
extern std::atomic<long long> g_launches;
inline void count_launch(long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Error word written by bounded device loops (never a trap).
enum DevErr : int { kDevOk = 0, kDevEighNoConv = 1, kDevNonFinite = 2, kDevTimeout = 3 };

// Record a device error; the first one recorded since the word was cleared wins, so that a root cause (a
// non-finite input) is not overwritten by what it causes downstream (an eigensolver that cannot converge).
__device__ __forceinline__ void raise_err(int *err, int code) { atomicCAS(err, (int)kDevOk, code); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum; every thread gets the result.  `red` holds >= blockDim.x/32 doubles.  Deterministic.
__device__ __forceinline__ double block_sum(double v, double *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w];
    return s;
}

__device__ __forceinline__ double block_max(double v, double *red) {
    v = warp_max(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double s = red[0];
    for (int w = 1; w < nw; ++w) s = fmax(s, red[w]);
    return s;
}

// ---------------------------------------------------------------------------- double-float arithmetic
// "Double-float": a value held as an unevaluated sum of two FP32 numbers (hi + lo, ~48 significant bits).  On
// GB300 an FP64 multiply-add issues at 1/64 of the FP32 rate, so FP64-accurate products of the mixed path run
// as double-float on the FP32 pipe (~12 FP32 operations per multiply-add).
// x ~ hi + lo with hi = x cut to 24 significant bits and lo the rest rounded to FP32, by integer operations
// (a double -> float conversion runs on the FP64 pipe).  Zero / subnormal / out-of-FP32-range values use the
// plain conversion.
__device__ __forceinline__ float2 split_df(double x) {
    const long long b = __double_as_longlong(x);
    const int ex = (int)((b >> 52) & 0x7FF);
    const int ef = ex - 1023 + 127;
    if (ex == 0 || ef < 53 || ef > 254) return make_float2((float)x, 0.f);   // |x| < 2^-74: lo negligible
    const unsigned sign = (unsigned)((unsigned long long)b >> 63) << 31;
    const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | (unsigned)((b >> 29) & 0x7FFFFF));
    const long long mlo = b & ((1LL << 29) - 1);   // value mlo 2^(ex - 1075)
    float lo = __ll2float_rn(mlo) * __uint_as_float((unsigned)(ef - 52) << 23);
    if (sign) lo = -lo;
    return make_float2(hi, lo);
}

// (sh, sl) += a * b for double-float a, b
__device__ __forceinline__ void df_fma(float &sh, float &sl, const float2 a, const float2 b) {
    const float p = __fmul_rn(a.x, b.x);
    const float e = fmaf(a.x, b.x, -p);
    const float c = fmaf(a.x, b.y, fmaf(a.y, b.x, e));
    const float t = __fadd_rn(sh, p);
    const float bp = __fsub_rn(t, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    sh = t;
    sl = __fadd_rn(sl, __fadd_rn(err, c));
}

// Two double-float multiply-adds at once on packed FP32 pairs (the f32x2 instructions of sm_100+: half the issue
// slots of two df_fma calls, bit-identical results): lane x of every float2 is one accumulation, lane y the
// other; (sh, sl) += a * (bh, bl) with a = (ah, al) shared by both.  The product error and cross terms are
// formed negated (fma with -a), so that no separate negation is needed.
__device__ __forceinline__ void df_fma2(float2 &sh, float2 &sl, float ah, float al, float2 bh, float2 bl) {
    const float2 nah = make_float2(-ah, -ah), nal = make_float2(-al, -al), m1 = make_float2(-1.f, -1.f);
    const float2 p = __fmul2_rn(make_float2(ah, ah), bh);
    const float2 en = __ffma2_rn(nah, bh, p);                          // -(p's rounding error)
    const float2 cn = __ffma2_rn(nah, bl, __ffma2_rn(nal, bh, en));    // -(error + cross terms)
    const float2 t = __fadd2_rn(sh, p);
    const float2 bp = __ffma2_rn(sh, m1, t);                           // t - sh
    const float2 err = __fadd2_rn(__ffma2_rn(__ffma2_rn(bp, m1, t), m1, sh), __ffma2_rn(bp, m1, p));
    sh = t;
    sl = __fadd2_rn(sl, __ffma2_rn(cn, m1, err));                      // sl + (err + c)
}

// 5 x 5 double-float tile update (h, l)[i][j] += x[i] y[j]: columns (0, 1) and (2, 3) as packed f32x2 pairs
__device__ __forceinline__ void df_tile5(float (&hh)[5][5], float (&ll)[5][5], const float2 *x, const float2 *y) {
    const float2 y01h = make_float2(y[0].x, y[1].x), y01l = make_float2(y[0].y, y[1].y);
    const float2 y23h = make_float2(y[2].x, y[3].x), y23l = make_float2(y[2].y, y[3].y);
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        float2 h0 = make_float2(hh[i][0], hh[i][1]), l0 = make_float2(ll[i][0], ll[i][1]);
        float2 h1 = make_float2(hh[i][2], hh[i][3]), l1 = make_float2(ll[i][2], ll[i][3]);
        df_fma2(h0, l0, x[i].x, x[i].y, y01h, y01l);
        df_fma2(h1, l1, x[i].x, x[i].y, y23h, y23l);
        hh[i][0] = h0.x; hh[i][1] = h0.y; ll[i][0] = l0.x; ll[i][1] = l0.y;
        hh[i][2] = h1.x; hh[i][3] = h1.y; ll[i][2] = l1.x; ll[i][3] = l1.y;
        df_fma(hh[i][4], ll[i][4], x[i], y[4]);
    }
}

// (hi, lo) += x with Knuth's two-sum (exact error term)
__device__ __forceinline__ void df_add(float &hi, float &lo, float x) {
    const float s = __fadd_rn(hi, x);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ float2 df_mul(const float2 a, const float2 b) {
    float h = 0.f, l = 0.f;
    df_fma(h, l, a, b);
    return make_float2(h, l);
}


// (hi + lo) 2^E as an FP64 number without the FP64 pipe (conversions and adds there run at 1/64 of the FP32
// rate on GB300): the pair is renormalised with an FP32 two-sum (|lo| <= ulp(hi) / 2), then sign, exponent and the
// significand (hi's 24 bits and lo's bits below them, in an int64) are assembled with integer operations.  Bits
// of lo more than 29 binades below hi's leading bit are truncated (< 1 ulp of the result).  Zero, subnormal and
// non-finite pairs and results outside the normal FP64 range take the FP64 route.
__host__ __device__ __forceinline__ double df_to_double(float hi, float lo, int E) {
#ifdef __CUDA_ARCH__
    const float s = __fadd_rn(hi, lo);
    const float bp = __fsub_rn(s, hi);
    const float l = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(lo, bp));
    const unsigned bh = __float_as_uint(s), bl = __float_as_uint(l);
#else
    const float s = hi + lo;
    const float bp = s - hi;
    const float l = (hi - (s - bp)) + (lo - bp);
    unsigned bh, bl;
    memcpy(&bh, &s, 4);
    memcpy(&bl, &l, 4);
#endif
    const int eh = (int)((bh >> 23) & 0xFFu), el = (int)((bl >> 23) & 0xFFu);
    int e = eh - 127 + 1023 + E;   // biased FP64 exponent of the leading bit
    if (eh == 0 || eh == 255 || el == 255 || (el == 0 && (bl & 0x7FFFFFu)) || e <= 1 || e >= 2046)
        return ldexp((double)s + (double)l, E);
    long long M = (long long)((bh & 0x7FFFFFu) | 0x800000u) << 29;
    if (el != 0) {
        const long long ml = (long long)((bl & 0x7FFFFFu) | 0x800000u);
        const int d = eh - el;   // >= 24 after the renormalisation
        const long long lv = d <= 29 ? ml << (29 - d) : (d < 54 ? ml >> (d - 29) : 0);
        if ((bh ^ bl) >> 31) M -= lv; else M += lv;
        if (M < (1LL << 52)) {   // hi a power of two, lo of the other sign
            M <<= 1;
            --e;
        }
    }
    const unsigned long long bits = ((unsigned long long)(bh >> 31) << 63) | ((unsigned long long)e << 52) |
                                    ((unsigned long long)M & ((1ULL << 52) - 1));
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double r;
    memcpy(&r, &bits, 8);
    return r;
#endif
}

// df_to_double without branches for the common case: finite hi and lo, hi zero or normal, lo zero or normal, the
// result exponent in the normal FP64 range.  special is set otherwise; the caller then takes df_to_double.
// The lo contribution is ((m_lo << 29) >> d) with d = e_hi - e_lo >= 24 after the renormalisation (one shift for
// both directions: exact for d <= 29, truncated beyond), so independent conversions interleave freely.
__host__ __device__ __forceinline__ double df_to_double_nb(float hi, float lo, int E, bool &special) {
#ifdef __CUDA_ARCH__
    const float s = __fadd_rn(hi, lo);
    const float bp = __fsub_rn(s, hi);
    const float l = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(lo, bp));
    const unsigned bh = __float_as_uint(s), bl = __float_as_uint(l);
#else
    const float s = hi + lo;
    const float bp = s - hi;
    const float l = (hi - (s - bp)) + (lo - bp);
    unsigned bh, bl;
    memcpy(&bh, &s, 4);
    memcpy(&bl, &l, 4);
#endif
    const int eh = (int)((bh >> 23) & 0xFFu), el = (int)((bl >> 23) & 0xFFu);
    int e = eh - 127 + 1023 + E;
    const unsigned long long mh = (unsigned long long)((bh & 0x7FFFFFu) | 0x800000u) << 29;
    const unsigned long long ml = el != 0 ? (unsigned long long)((bl & 0x7FFFFFu) | 0x800000u) << 29 : 0ULL;
    const int d = max(0, min(eh - el, 63));
    const unsigned long long lv = ml >> d;
    unsigned long long M = ((bh ^ bl) >> 31) ? mh - lv : mh + lv;
    const bool low = M < (1ULL << 52);   // hi a power of two, lo of the other sign
    M = low ? M << 1 : M;
    e = low ? e - 1 : e;
    special = eh == 255 || el == 255 || (el == 0 && (bl & 0x7FFFFFu)) || (eh != 0 && (e <= 1 || e >= 2046));
    const unsigned long long sign = (unsigned long long)(bh >> 31) << 63;
    const unsigned long long bits = eh == 0 ? sign : sign | ((unsigned long long)e << 52) | (M & ((1ULL << 52) - 1));
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double r;
    memcpy(&r, &bits, 8);
    return r;
#endif
}

// (h + l) g 2^E for a double-float g: the product in double-float on the FP32 pipe, then integer assembly
__device__ __forceinline__ double df_to_double_mul(float h, float l, float2 g, int E) {
    float ph = 0.f, pl = 0.f;
    df_fma(ph, pl, make_float2(h, l), g);
    return df_to_double(ph, pl, E);
}

// h + l in FP64 on the FP64 pipe (kernels whose FP32 pipe is the bottleneck; df_to_double where FP64 is)
__device__ __forceinline__ double df_val(float h, float l) { return (double)h + (double)l; }

// Element copies global -> shared (4 or 8 bytes) that stay in flight together: a staging loop issues all of its
// copies before any completes, instead of one load latency per element.  src_bytes = 0 zero-fills.
__device__ __forceinline__ void cpa_elem(void *dst, const void *src, int bytes, int src_bytes = -1) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    const int sb = src_bytes < 0 ? bytes : src_bytes;
    if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(sb) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(sb) : "memory");
}
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }


// ------------------------------------------------------------------------------------ grouped FP64 GEMM
// C[M x N] = alpha * opA(A)[M x K] * opB(B)[K x N] + beta * C, every matrix row-major.
//   transA = 0: A(m,k) = A[arow(m) * lda + acol(k)],  transA = 1: A(m,k) = A[acol(k) * lda + m]
//   transB = 0: B(k,n) = B[brow(k) * ldb + bcol(n)],  transB = 1: B(k,n) = B[bcol(n) * ldb + brow(k)]
//   arow(m) = a_rows ? a_rows[m] : m;  acol(k) = k_idx_a ? k_idx_a[k] : k
//   brow(k) = k_idx_b ? k_idx_b[k] : k;  bcol(n) = n_idx_b ? n_idx_b[n] : n
//   C(m,n) at C[m * ldc + ccol(n)], ccol(n) = n_idx_c ? n_idx_c[n] : n
//   atomic = 1: C(m,n) += alpha * acc with atomicAdd (beta ignored).
struct GemmDesc {
    int M, N, K;
    int transA, transB, atomic;
    long long lda, ldb, ldc;
    const double *A;
    const double *B;
    double *C;
    double alpha, beta;
    const int *a_rows;
    const int *k_idx_a;
    const int *k_idx_b;
    const int *n_idx_b;
    const int *n_idx_c;
    int *ea;   // row scales of A and column scales of B (exact-slice tensor-core GEMM; set by its prepare step)
    int *eb;
};

// Host-side batch of GEMM problems: descriptors and per-problem tile offsets live in device memory.
struct GemmBatch {
    std::vector<GemmDesc> h;
    GemmDesc *d_desc = nullptr;
    long long *d_tile0 = nullptr;
    long long tiles = 0;
    long long *d_tile0_df = nullptr;   // tile offsets of the double-float kernel's shape
    long long tiles_df = 0;
    int df_shape = 0;                  // 0: 64 x 64, 1: 80 x 80, 2: 48 x 80, 3: 80 x 48, 4: 48 x 48
    int df_rule = 0;                   // the shape the padded-work rule chose at upload
    void add(const GemmDesc &g) { h.push_back(g); }
};

cudaError_t gemm_batch_upload(GemmBatch &b);
// the double-float kernel's tile shape of an uploaded batch: 0 64x64, 1 80x80, 2 48x80, 3 80x48, 4 48x48
cudaError_t gemm_batch_set_df_shape(GemmBatch &b, int shape);
cudaError_t gemm_batch_run(const GemmBatch &b, cudaStream_t s);
// the same batch in double-float arithmetic on the FP32 pipe (~2^-44 relative)
cudaError_t gemm_batch_run_df(const GemmBatch &b, cudaStream_t s);
void gemm_batch_free(GemmBatch &b);

inline GemmDesc gemm(int M, int N, int K, const double *A, long long lda, int tA, const double *B,
                     long long ldb, int tB, double *C, long long ldc, double alpha = 1.0, double beta = 0.0) {
    GemmDesc g{};
    g.M = M; g.N = N; g.K = K;
    g.A = A; g.lda = lda; g.transA = tA;
    g.B = B; g.ldb = ldb; g.transB = tB;
    g.C = C; g.ldc = ldc;
    g.alpha = alpha; g.beta = beta;
    return g;
}

// ------------------------------------------------------------------------------------- batched eigh
// One symmetric matrix A (n x n, row-major, leading dimension lda) to diagonalise.  A is overwritten.
// n_dev (optional): device int with the actual order (<= n) used instead of n; the rest is left alone.
// Output: w (decreasing eigenvalues), Zt (eigenvector mu in row mu, leading dimension ldz).
// zwork: n x n scratch (column-major eigenvector accumulation).
struct EighDesc {
    double *A;
    long long lda;
    int n;
    const int *n_dev;
    double *w;
    double *Zt;
    long long ldz;
    double *zwork;   // n x n scratch (the mixed small Jacobi keeps its FP32 first-stage vectors here)
    double *d;     // n scratch (diagonal)
    double *e;     // n scratch (sub-diagonal)
    double *tau;   // n scratch (Householder scalars)
};

// Diagonalise every matrix of the batch; err (device int) receives kDevEighNoConv on an iteration cap.
cudaError_t eigh_batched(const EighDesc *d_desc, int batch, int n_max, int rows_split, int *err,
                         cudaStream_t s);

}  // namespace osv
